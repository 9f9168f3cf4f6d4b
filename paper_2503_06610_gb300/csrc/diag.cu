// diag.cu -- field conversion, population initialisation and the FP64 global
// diagnostics (mass, lattice Frank energy, |u| and |n| extrema, NaN count,
// skyrmion-tube centroid sums) of the hybrid LB + FD library.
#include "diag_sum.cuh"

namespace nh {

namespace {

template <typename Real>
__global__ void load_fields_kernel(const double* __restrict__ n, const double* __restrict__ u,
                                   const double* __restrict__ rho, Real* dn, Real* du, Real* drho, int N)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const double a = n[s], b = n[N + s], c = n[2 * N + s];
    const double inv = 1.0 / sqrt(a * a + b * b + c * c);
    dn[s] = Real(a * inv);
    dn[N + s] = Real(b * inv);
    dn[2 * N + s] = Real(c * inv);
    for (int k = 0; k < 3; ++k) du[k * N + s] = u ? Real(u[k * N + s]) : Real(0);
    drho[s] = rho ? Real(rho[s]) : Real(1);
}

template <typename Real>
__global__ void store_vec_kernel(const Real* __restrict__ src, double* __restrict__ dst, int64_t count)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dst[i] = (double)src[i];
}

template <typename Real, typename Store, bool Shifted>
__global__ void init_populations_kernel(const Real* __restrict__ rho, const Real* __restrict__ u, Store* f,
                                        const float* scale, int N)
{
    NH_D3Q19_TABLES
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const float sc = sizeof(Store) == 2 ? scale[0] : 1.f;
    const Real r = rho[s];
    const Real ux = u[s], uy = u[N + s], uz = u[2 * N + s];
    const Real uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const Real w = d3q19_w<Real>(i);
        const Real eu = Real(EX[i]) * ux + Real(EY[i]) * uy + Real(EZ[i]) * uz;
        Real feq = w * r * (Real(3) * eu + Real(4.5) * eu * eu - Real(1.5) * uu);
        feq += Shifted ? w * (r - Real(1)) : w * r;
        Codec<Store, Real>::store(f + (size_t)i * N + s, feq, sc);
    }
}

template <typename Store>
__global__ void decode_plane_kernel(const Store* __restrict__ f, double* __restrict__ dst, int N, const float* scale)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    if constexpr (sizeof(Store) == 2) {
        dst[s] = (double)Codec<Store, float>::load(f + s, 1.f / scale[0]);
    } else {
        dst[s] = (double)f[s];
    }
}

template <typename Store>
__global__ void encode_plane_kernel(const double* __restrict__ src, Store* __restrict__ f, int N, const float* scale)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    if constexpr (sizeof(Store) == 2) {
        Codec<Store, float>::store(f + s, (float)src[s], scale[0]);
    } else {
        f[s] = (Store)src[s];
    }
}

// Initial power-of-two scale of a 16-bit store: from the largest equilibrium
// population of the initial state and half the largest body force (the size of
// the first Guo source), so that both start near 2^kScaleHeadroomLog2.
__global__ void scale_probe_kernel(const float* __restrict__ rho, const float* __restrict__ u,
                                   const float* __restrict__ F, float gx, float gy, float gz, int N, unsigned* ctrl)
{
    NH_D3Q19_TABLES
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    float m = 0.f;
    if (s < N) {
        const float r = rho[s];
        const float ux = u[s], uy = u[N + s], uz = u[2 * N + s];
        const float uu = ux * ux + uy * uy + uz * uz;
        for (int i = 0; i < 19; ++i) {
            const float w = d3q19_w<float>(i);
            const float eu = EX[i] * ux + EY[i] * uy + EZ[i] * uz;
            m = fmaxf(m, fabsf(w * r * (3.f * eu + 4.5f * eu * eu - 1.5f * uu) + w * (r - 1.f)));
        }
        const float fx = F[s] + r * gx, fy = F[N + s] + r * gy, fz = F[2 * N + s] + r * gz;
        m = fmaxf(m, 0.5f * sqrtf(fx * fx + fy * fy + fz * fz));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(reinterpret_cast<int*>(&ctrl[0]), __float_as_int(m));
}

__global__ void scale_set_kernel(float* scales, unsigned* ctrl)
{
    const float m = __uint_as_float(ctrl[0]);
    float t = 1.f;
    if (m > 0.f && isfinite(m)) {
        int e;
        frexpf(m, &e);
        int k = kScaleHeadroomLog2 - e;
        k = k < -120 ? -120 : (k > 120 ? 120 : k);
        t = ldexpf(1.f, k);
    }
    scales[0] = scales[1] = scales[2] = t;
    ctrl[0] = 0u;
    ctrl[1] = 0u;
}

// ------------------------------------------------------------------ diagnostics

using dsum::DIAG_FIXED;
using dsum::DIAG_THREADS;
using dsum::link_energy;
using dsum::warp_max;
using dsum::warp_min;
using dsum::warp_sum;
using dsum::warp_tube_accumulate;

__device__ __forceinline__ int nearest_tube(const DiagArgs& a, const float (*txy)[2], int T, int x, int y)
{
    return dsum::nearest_tube(a.g, &a.tubes[0][0], txy, T, x, y);
}
template <typename Real>
__device__ __forceinline__ void tube_values(const DiagArgs& a, int x, int y, Real wsum, Real v[5])
{
    dsum::tube_values(a.g, a.trig, x, y, wsum, v);
}
template <typename Real>
__device__ __forceinline__ void diag_block_partials(const DiagArgs& a, Real mass_t, Real energy_t, Real max_u,
                                                    Real min_nn, Real max_nn, int bad,
                                                    const Real (*tube_acc)[NH_MAX_TUBES * 5], int T)
{
    dsum::block_partials(a.partials, a.lbpart, a.lbp_blocks, mass_t, energy_t, max_u, min_nn, max_nn, bad, tube_acc, T);
}

// Work item = (x, y) column x a chunk of kDiagChunk layers; one thread per item
// (grid-stride; the items of a warp share the chunk, so z-branches are uniform).
// A thread marches up its chunk: the director of the next layer is loaded one
// site ahead and is both the z+1 link partner and the next centre, the x+1 and
// y+1 partners are branch-free loads, and the loop is unrolled so that several
// sites' loads are in flight.  Per-site terms are summed over the chunk in the
// build's precision (Real) over a thread's items, then in FP64 across threads.
// Tube sums use the item's weight sum_z (1 - n_z)/2, the column's nearest
// previous centroid (FP32 periodic distance with an FP64 tie check), the
// FP64 sin/cos tables of the column position, a warp sum and a per-warp
// shared-memory sum in Real per owner, and FP64 accumulation across warps.
constexpr int kDiagChunk = 8;
// Reading the director alone (NOnly) leaves the loop short of loads in
// flight per site, so longer chunks lose little latency hiding, and the
// column's tube work (nearest centroid, sin/cos) is then shared by 16 layers.
constexpr int kDiagChunkN = 16;

template <typename Real>
__device__ __forceinline__ void load3(const Real* __restrict__ n, int N, int s, Real out[3])
{
    out[0] = __ldg(n + s);
    out[1] = __ldg(n + N + s);
    out[2] = __ldg(n + 2 * N + s);
}

// NOnly: the populations, u and rho were summed by the LB launch that wrote
// them (lb.cu, a.lbpart); only the director is read here.
template <typename Real, typename Store, bool F3, bool Solid, bool NOnly = false>
__global__ void __launch_bounds__(DIAG_THREADS, (sizeof(Real) == 4 && !F3 && !Solid) ? 5 : 1)
    diag_kernel(const DiagArgs a)
{
    const Geom g = a.g;
    const int N = g.N;
    const int cols = g.nx * g.ny;
    constexpr int kChunk = NOnly ? kDiagChunkN : kDiagChunk;
    const int chunks = (g.nz + kChunk - 1) / kChunk;
    const int items = cols * chunks;
    const Store* __restrict__ f = static_cast<const Store*>(a.f);
    const Real* __restrict__ n = static_cast<const Real*>(a.n);
    const Real* __restrict__ u = static_cast<const Real*>(a.u);
    const Real* __restrict__ rho = static_cast<const Real*>(a.rho);
    const float inv_scale = sizeof(Store) == 2 ? 1.f / a.scale[0] : 1.f;
    const Real K = Real(a.K), q0 = Real(a.q0), W0 = Real(a.W0);
    const Real site_const = Real(0.5) * K * q0 * q0;
    const bool homeo = g.walls && g.anchoring == NH_ANCHOR_HOMEOTROPIC;
    const unsigned char* __restrict__ sm = a.solid;
    const int T = a.n_tubes;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // tube sums per warp in the build's precision (lane 0 of each warp owns its
    // row: no atomics); combined in FP64 across warps and blocks
    __shared__ Real tube_acc[DIAG_THREADS / 32][NH_MAX_TUBES * 5];
    __shared__ float tube_xy[NH_MAX_TUBES][2];
    for (int k = threadIdx.x; k < (DIAG_THREADS / 32) * NH_MAX_TUBES * 5; k += blockDim.x)
        (&tube_acc[0][0])[k] = Real(0);
    for (int k = threadIdx.x; k < T; k += blockDim.x) {
        tube_xy[k][0] = (float)a.tubes[k][0];
        tube_xy[k][1] = (float)a.tubes[k][1];
    }
    __syncthreads();

    Real mass_t = 0, energy_t = 0;  // this thread's sums over its items (build precision)
    Real max_u = 0, min_nn = Real(1e30), max_nn = 0;
    int bad = 0;
    for (int base = blockIdx.x * blockDim.x; base < items; base += gridDim.x * blockDim.x) {
        const int item = base + threadIdx.x;
        const bool valid = item < items;
        Real wsum = 0;
        int x = 0, y = 0;
        if (valid) {
            const int col = item % cols;
            const int z0 = (item / cols) * kChunk;
            const int z1 = min(z0 + kChunk, g.nz);
            x = col % g.nx;
            y = col / g.nx;
            const int colx = (x + 1 == g.nx ? 0 : x + 1) + g.nx * y;
            const int coly = x + g.nx * (y + 1 == g.ny ? 0 : y + 1);
            const int colxm = (x == 0 ? g.nx - 1 : x - 1) + g.nx * y;
            const int colym = x + g.nx * (y == 0 ? g.ny - 1 : y - 1);
            Real msum = 0, esum = 0;
            Real c[3];
            load3(n, N, col + cols * z0, c);
            Real cl[3] = {c[0], c[1], c[2]};  // director one layer below (three-constant gradient)
            if (F3) {
                if (z0 > 0) {
                    load3(n, N, col + cols * (z0 - 1), cl);
                } else if (!g.walls) {
                    load3(n, N, col + cols * (g.nz - 1), cl);
                } else if (homeo) {
                    cl[0] = Real(0);
                    cl[1] = Real(0);
                    cl[2] = Real(1);
                }
            }
            if (g.walls && z0 == 0 && !(Solid && sm[col])) {
                // link from the lower ghost layer to the first fluid layer
                Real m[3] = {c[0], c[1], c[2]};
                if (homeo) {
                    m[0] = Real(0);
                    m[1] = Real(0);
                    m[2] = Real(1);
                }
                esum += link_energy(m, c, 2, K, q0);
            }
#pragma unroll 4
            for (int z = z0; z < z1; ++z) {
                const int s = col + cols * z;
                Real cn[3];
                if (z + 1 < g.nz) {
                    load3(n, N, s + cols, cn);
                } else if (!g.walls) {
                    load3(n, N, col, cn);  // periodic in z
                } else if (homeo) {
                    cn[0] = Real(0);
                    cn[1] = Real(0);
                    cn[2] = Real(1);
                } else {
                    cn[0] = c[0];
                    cn[1] = c[1];
                    cn[2] = c[2];
                }
                Real mx[3], my[3];
                load3(n, N, colx + cols * z, mx);
                load3(n, N, coly + cols * z, my);
                Real fs = 0, u0 = 0, u1 = 0, u2 = 0, r = 1;
                if (!NOnly) {
#pragma unroll
                    for (int i = 0; i < 19; ++i) fs += Codec<Store, Real>::load(f + (size_t)i * N + s, inv_scale);
                    u0 = __ldg(u + s);
                    u1 = __ldg(u + N + s);
                    u2 = __ldg(u + 2 * N + s);
                    r = __ldg(rho + s);
                }
                // obstacles: sums over fluid sites, links with at least one fluid end
                bool sol = false, solx = false, soly = false, solz = false;
                if (Solid) {
                    sol = sm[s] != 0;
                    solx = sm[colx + cols * z] != 0;
                    soly = sm[coly + cols * z] != 0;
                    solz = z + 1 < g.nz ? sm[s + cols] != 0 : (!g.walls ? sm[col] != 0 : true);
                }
                Real e = (sol && solx) ? Real(0) : link_energy(c, mx, 0, K, q0);
                if (!(sol && soly)) e += link_energy(c, my, 1, K, q0);
                if (!(sol && solz)) e += link_energy(c, cn, 2, K, q0);
                esum += e;
                if (!sol) {
                    msum += fs;
                    esum += site_const - Real(0.5) * W0 * c[2] * c[2];
                    if (F3) {
                        // three-constant correction with the central gradient
                        Real mxm[3], mym[3];
                        load3(n, N, colxm + cols * z, mxm);
                        load3(n, N, colym + cols * z, mym);
                        Real G[3][3], dfdn[3], P[3][3];
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            G[0][k] = Real(0.5) * (mx[k] - mxm[k]);
                            G[1][k] = Real(0.5) * (my[k] - mym[k]);
                            G[2][k] = Real(0.5) * (cn[k] - cl[k]);
                        }
                        esum += frank3_site(c, G, Real(a.kd1), Real(a.kd2), Real(a.kd3), q0, dfdn, P);
                    }
                    const Real umag = sqrt(u0 * u0 + u1 * u1 + u2 * u2);
                    const Real nmag = dsum::norm3(c);
                    max_u = max(max_u, umag);
                    min_nn = min(min_nn, nmag);
                    max_nn = max(max_nn, nmag);
                    // a site counts once for a bad director and once for a bad u, rho or population sum
                    bad += !isfinite(nmag) ? 1 : 0;
                    if (!NOnly && (!isfinite(umag) || !isfinite(r) || !isfinite(fs))) bad += 1;
                    wsum += Real(0.5) * (Real(1) - c[2]);
                }  // fluid site
                if (F3) {
                    cl[0] = c[0];
                    cl[1] = c[1];
                    cl[2] = c[2];
                }
                c[0] = cn[0];
                c[1] = cn[1];
                c[2] = cn[2];
            }
            mass_t += msum;
            energy_t += esum;
        }
        if (T > 0) {
            int owner = -1;
            Real v[5] = {0, 0, 0, 0, 0};
            if (valid) {
                owner = nearest_tube(a, tube_xy, T, x, y);
                tube_values(a, x, y, wsum, v);
            }
            warp_tube_accumulate(owner, v, lane, tube_acc[wid]);
        }
    }
    diag_block_partials(a, mass_t, energy_t, max_u, min_nn, max_nn, bad, tube_acc, T);
}

// Two-column variant of the plain path (one-constant energy, no obstacles,
// nx even): an item is the x-pair of columns (x, x + 1), x even, times a
// chunk of kDiagPairChunk layers.  Populations, n, u and rho of the pair are
// read as one 2-vector each (s even, so the vectors are aligned), the x + 1
// partner of the first site is the second site, and only the second site's
// x + 1 partner is a scalar load: half the load instructions per site of the
// one-column kernel, twice the bytes in flight per thread.  The same sums.
constexpr int kDiagPairChunk = 4;
constexpr int kDiagPairChunkN = 16;  // director only (NOnly), as kDiagChunkN

template <typename Real>
struct Pair;
template <>
struct Pair<float> {
    using T = float2;
};
template <>
struct Pair<double> {
    using T = double2;
};

template <typename Real>
__device__ __forceinline__ void load3_pair(const Real* __restrict__ n, int N, int s, Real p[3], Real q[3])
{
    using V = typename Pair<Real>::T;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const V v = __ldg(reinterpret_cast<const V*>(n + k * N + s));
        p[k] = v.x;
        q[k] = v.y;
    }
}

// Two consecutive populations (sites s, s + 1 of one plane), decoded as Codec does.
template <typename Real>
__device__ __forceinline__ void pop_pair(const Real* p, float, Real& a, Real& b)
{
    const typename Pair<Real>::T v = __ldg(reinterpret_cast<const typename Pair<Real>::T*>(p));
    a = v.x;
    b = v.y;
}
__device__ __forceinline__ void pop_pair(const __half* p, float inv_scale, float& a, float& b)
{
    const __half2 h = __ldg(reinterpret_cast<const __half2*>(p));
    a = __low2float(h) * inv_scale;
    b = __high2float(h) * inv_scale;
}
__device__ __forceinline__ void pop_pair(const __nv_bfloat16* p, float inv_scale, float& a, float& b)
{
    const __nv_bfloat162 h = __ldg(reinterpret_cast<const __nv_bfloat162*>(p));
    a = __low2float(h) * inv_scale;
    b = __high2float(h) * inv_scale;
}

template <typename Real, typename Store, bool NOnly = false>
__global__ void __launch_bounds__(DIAG_THREADS, sizeof(Real) == 4 ? 4 : 1) diag_pair_kernel(const DiagArgs a)
{
    const Geom g = a.g;
    const int N = g.N;
    const int cols = g.nx * g.ny;
    const int hx = g.nx >> 1;  // pairs per row
    const int pcols = hx * g.ny;
    constexpr int kChunk = NOnly ? kDiagPairChunkN : kDiagPairChunk;
    const int chunks = (g.nz + kChunk - 1) / kChunk;
    const int items = pcols * chunks;
    const Store* __restrict__ f = static_cast<const Store*>(a.f);
    const Real* __restrict__ n = static_cast<const Real*>(a.n);
    const Real* __restrict__ u = static_cast<const Real*>(a.u);
    const Real* __restrict__ rho = static_cast<const Real*>(a.rho);
    const float inv_scale = sizeof(Store) == 2 ? 1.f / a.scale[0] : 1.f;
    const Real K = Real(a.K), q0 = Real(a.q0), W0 = Real(a.W0);
    const Real site_const = Real(0.5) * K * q0 * q0;
    const bool homeo = g.walls && g.anchoring == NH_ANCHOR_HOMEOTROPIC;
    const int T = a.n_tubes;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __shared__ Real tube_acc[DIAG_THREADS / 32][NH_MAX_TUBES * 5];
    __shared__ float tube_xy[NH_MAX_TUBES][2];
    for (int k = threadIdx.x; k < (DIAG_THREADS / 32) * NH_MAX_TUBES * 5; k += blockDim.x)
        (&tube_acc[0][0])[k] = Real(0);
    for (int k = threadIdx.x; k < T; k += blockDim.x) {
        tube_xy[k][0] = (float)a.tubes[k][0];
        tube_xy[k][1] = (float)a.tubes[k][1];
    }
    __syncthreads();

    Real mass_t = 0, energy_t = 0;
    Real max_u = 0, min_nn = Real(1e30), max_nn = 0;
    int bad = 0;
    for (int base = blockIdx.x * blockDim.x; base < items; base += gridDim.x * blockDim.x) {
        const int item = base + threadIdx.x;
        const bool valid = item < items;
        Real wsum0 = 0, wsum1 = 0;
        int x = 0, y = 0;
        if (valid) {
            const int pc = item % pcols;
            const int z0 = (item / pcols) * kChunk;
            const int z1 = min(z0 + kChunk, g.nz);
            x = 2 * (pc % hx);
            y = pc / hx;
            const int col = x + g.nx * y;
            const int colx2 = (x + 2 == g.nx ? 0 : x + 2) + g.nx * y;  // x + 1 partner of the second site
            const int coly = x + g.nx * (y + 1 == g.ny ? 0 : y + 1);
            Real msum = 0, esum = 0;
            Real c0[3], c1[3];
            load3_pair(n, N, col + cols * z0, c0, c1);
            if (g.walls && z0 == 0) {
                // links from the lower ghost layer to the first fluid layer
                Real m0[3] = {c0[0], c0[1], c0[2]}, m1[3] = {c1[0], c1[1], c1[2]};
                if (homeo) {
                    m0[0] = m0[1] = m1[0] = m1[1] = Real(0);
                    m0[2] = m1[2] = Real(1);
                }
                esum += link_energy(m0, c0, 2, K, q0);
                esum += link_energy(m1, c1, 2, K, q0);
            }
#pragma unroll 2
            for (int z = z0; z < z1; ++z) {
                const int s = col + cols * z;
                Real n0[3], n1[3];  // z + 1 partners
                if (z + 1 < g.nz) {
                    load3_pair(n, N, s + cols, n0, n1);
                } else if (!g.walls) {
                    load3_pair(n, N, col, n0, n1);  // periodic in z
                } else if (homeo) {
                    n0[0] = n0[1] = n1[0] = n1[1] = Real(0);
                    n0[2] = n1[2] = Real(1);
                } else {
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        n0[k] = c0[k];
                        n1[k] = c1[k];
                    }
                }
                Real y0[3], y1[3], x2[3];
                load3_pair(n, N, coly + cols * z, y0, y1);
                load3(n, N, colx2 + cols * z, x2);
                Real fs0 = 0, fs1 = 0;
                Real ua[3] = {0, 0, 0}, ub[3] = {0, 0, 0};
                typename Pair<Real>::T r;
                r.x = r.y = Real(1);
                if (!NOnly) {
#pragma unroll
                    for (int i = 0; i < 19; ++i) {
                        Real p0, p1;
                        pop_pair(f + (size_t)i * N + s, inv_scale, p0, p1);
                        fs0 += p0;
                        fs1 += p1;
                    }
                    load3_pair(u, N, s, ua, ub);
                    r = __ldg(reinterpret_cast<const typename Pair<Real>::T*>(rho + s));
                }
                Real e = link_energy(c0, c1, 0, K, q0);
                e += link_energy(c0, y0, 1, K, q0);
                e += link_energy(c0, n0, 2, K, q0);
                e += link_energy(c1, x2, 0, K, q0);
                e += link_energy(c1, y1, 1, K, q0);
                e += link_energy(c1, n1, 2, K, q0);
                esum += e;
                msum += fs0 + fs1;
                esum += Real(2) * site_const - Real(0.5) * W0 * (c0[2] * c0[2] + c1[2] * c1[2]);
                const Real umag0 = dsum::norm3(ua);
                const Real umag1 = dsum::norm3(ub);
                const Real nmag0 = dsum::norm3(c0);
                const Real nmag1 = dsum::norm3(c1);
                max_u = max(max_u, max(umag0, umag1));
                min_nn = min(min_nn, min(nmag0, nmag1));
                max_nn = max(max_nn, max(nmag0, nmag1));
                bad += (!isfinite(nmag0) ? 1 : 0) + (!isfinite(nmag1) ? 1 : 0);
                if (!NOnly) {
                    if (!isfinite(umag0) || !isfinite(r.x) || !isfinite(fs0)) bad += 1;
                    if (!isfinite(umag1) || !isfinite(r.y) || !isfinite(fs1)) bad += 1;
                }
                wsum0 += Real(0.5) * (Real(1) - c0[2]);
                wsum1 += Real(0.5) * (Real(1) - c1[2]);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    c0[k] = n0[k];
                    c1[k] = n1[k];
                }
            }
            mass_t += msum;
            energy_t += esum;
        }
        if (T > 0) {
#pragma unroll 1
            for (int j = 0; j < 2; ++j) {
                int owner = -1;
                Real v[5] = {0, 0, 0, 0, 0};
                if (valid) {
                    owner = nearest_tube(a, tube_xy, T, x + j, y);
                    tube_values(a, x + j, y, j ? wsum1 : wsum0, v);
                }
                warp_tube_accumulate(owner, v, lane, tube_acc[wid]);
            }
        }
    }
    diag_block_partials(a, mass_t, energy_t, max_u, min_nn, max_nn, bad, tube_acc, T);
}

// One block per reduced value: each thread combines a strided subset of the
// block partials (stored value-major, so the loads are contiguous), then a
// fixed shared-memory tree combines the threads, so the result is
// deterministic.  Spread over V blocks because FP64 throughput per SM is low.
constexpr int kFinalThreads = 256;
constexpr int kFinalLoads = 8;
__global__ void __launch_bounds__(kFinalThreads) diag_final_kernel(const double* __restrict__ partials,
                                                                   double* __restrict__ result, int blocks, int V)
{
    const int k = blockIdx.x;
    if (k >= V) return;
    const int kind = (k == 2 || k == 4) ? 1 : (k == 3 ? 2 : 0);  // 0 sum, 1 max, 2 min
    const double id = kind == 2 ? 1e300 : 0.0;
    double acc = id;
    // kFinalLoads loads in flight per thread, then combined in a fixed order
    auto fold = [&](const double* __restrict__ src, int count) {
        for (int b0 = threadIdx.x; b0 < count; b0 += kFinalLoads * kFinalThreads) {
            double v[kFinalLoads];
#pragma unroll
            for (int j = 0; j < kFinalLoads; ++j) {
                const int b = b0 + j * kFinalThreads;
                v[j] = b < count ? __ldg(src + b) : id;
            }
#pragma unroll
            for (int j = 0; j < kFinalLoads; ++j)
                acc = kind == 0 ? acc + v[j] : (kind == 1 ? fmax(acc, v[j]) : fmin(acc, v[j]));
        }
    };
    fold(partials + (size_t)k * blocks, blocks);
    __shared__ double sh[kFinalThreads];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kFinalThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const double w = sh[threadIdx.x + o];
            const double a = sh[threadIdx.x];
            sh[threadIdx.x] = kind == 0 ? a + w : (kind == 1 ? fmax(a, w) : fmin(a, w));
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) result[k] = sh[0];
}

// sin / cos of 2 pi x / nx and 2 pi y / ny in FP64, laid out [sx | cx | sy | cy].
__global__ void trig_table_kernel(double* t, int nx, int ny)
{
    const double twopi = 6.283185307179586476925286766559;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nx + ny; i += gridDim.x * blockDim.x) {
        double sv, cv;
        if (i < nx) {
            sincos(twopi * i / nx, &sv, &cv);
            t[i] = sv;
            t[nx + i] = cv;
        } else {
            const int j = i - nx;
            sincos(twopi * j / ny, &sv, &cv);
            t[2 * nx + j] = sv;
            t[2 * nx + ny + j] = cv;
        }
    }
}

// max over sites of |n - snap| (the largest change of the director since the
// snapshot), then snap <- n.  Per-block maxima go to partial[block].
template <typename Real>
__global__ void director_change_kernel(const Real* __restrict__ n, Real* __restrict__ snap, double* partial, int N)
{
    double m = 0.0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
        double d2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            const Real v = n[(size_t)a * N + s];
            const double d = (double)v - (double)snap[(size_t)a * N + s];
            d2 += d * d;
            snap[(size_t)a * N + s] = v;
        }
        m = fmax(m, sqrt(d2));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ double wm[8];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = fmax(b, wm[w]);
        partial[blockIdx.x] = b;
    }
}

__global__ void max_final_kernel(const double* __restrict__ partial, double* __restrict__ out, int blocks)
{
    double m = 0.0;
    for (int b = threadIdx.x; b < blocks; b += 32) m = fmax(m, partial[b]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) *out = m;
}

// Average of the four images of n under rotations by 90 degrees about the
// z axis through the site (c, c), c = nx / 2 (requires nx == ny): with
// X = x - c, Y = y - c and R n = (-n_y, n_x, n_z),
//   out(p) = 1/4 sum_k R^k n(R^-k p),  R^-1 (X, Y) = (Y, -X),
// then normalised.
template <typename Real>
__global__ void symmetrize_c4_kernel(const Real* __restrict__ n, Real* __restrict__ out, int nx, int nz)
{
    const int N = nx * nx * nz;
    const int c = nx / 2;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
        const int x = s % nx, y = (s / nx) % nx, z = s / (nx * nx);
        const int X = x - c, Y = y - c;
        const int px[4] = {x, c + Y, c - X, c - Y};
        const int py[4] = {y, c - X, c - Y, c + X};
        double v[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < 4; ++k) {
            const int xs = ((px[k] % nx) + nx) % nx, ys = ((py[k] % nx) + nx) % nx;
            const size_t q = (size_t)xs + (size_t)nx * ((size_t)ys + (size_t)nx * z);
            const double a = (double)n[q], b = (double)n[(size_t)N + q], w = (double)n[2 * (size_t)N + q];
            if (k == 0) { v[0] += a; v[1] += b; }
            if (k == 1) { v[0] -= b; v[1] += a; }
            if (k == 2) { v[0] -= a; v[1] -= b; }
            if (k == 3) { v[0] += b; v[1] -= a; }
            v[2] += w;
        }
        const double inv = 1.0 / dsum::norm3(v);
        out[s] = (Real)(v[0] * inv);
        out[(size_t)N + s] = (Real)(v[1] * inv);
        out[2 * (size_t)N + s] = (Real)(v[2] * inv);
    }
}

inline int blocks_for(int64_t n) { return (int)((n + 255) / 256); }

}  // namespace

template <typename Real>
cudaError_t launch_symmetrize_c4(const Real* n, Real* out, int nx, int nz, cudaStream_t st)
{
    const int N = nx * nx * nz;
    int blocks = blocks_for(N);
    if (blocks > 4096) blocks = 4096;
    symmetrize_c4_kernel<Real><<<blocks, 256, 0, st>>>(n, out, nx, nz);
    return cudaGetLastError();
}
template cudaError_t launch_symmetrize_c4<double>(const double*, double*, int, int, cudaStream_t);
template cudaError_t launch_symmetrize_c4<float>(const float*, float*, int, int, cudaStream_t);

template <typename Real>
cudaError_t launch_director_change(const Real* n, Real* snap, double* partial, double* out, int N, cudaStream_t st)
{
    int blocks = blocks_for(N);
    if (blocks > diag_blocks()) blocks = diag_blocks();
    director_change_kernel<Real><<<blocks, 256, 0, st>>>(n, snap, partial, N);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    max_final_kernel<<<1, 32, 0, st>>>(partial, out, blocks);
    return cudaGetLastError();
}
template cudaError_t launch_director_change<double>(const double*, double*, double*, double*, int, cudaStream_t);
template cudaError_t launch_director_change<float>(const float*, float*, double*, double*, int, cudaStream_t);

int diag_num_values(int n_tubes) { return DIAG_FIXED + 5 * n_tubes; }
int diag_blocks() { return 5 * 152; }

template <typename Real>
cudaError_t launch_load_fields(const double* n, const double* u, const double* rho, Real* dn, Real* du, Real* drho,
                               int N, cudaStream_t st)
{
    load_fields_kernel<Real><<<blocks_for(N), 256, 0, st>>>(n, u, rho, dn, du, drho, N);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_store_vec(const Real* src, double* dst, int64_t count, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    store_vec_kernel<Real><<<blocks_for(count), 256, 0, st>>>(src, dst, count);
    return cudaGetLastError();
}

template <typename Real, typename Store>
cudaError_t launch_init_populations(const Real* rho, const Real* u, Store* f, const float* scale, int N, bool shifted,
                                    cudaStream_t st)
{
    if (shifted)
        init_populations_kernel<Real, Store, true><<<blocks_for(N), 256, 0, st>>>(rho, u, f, scale, N);
    else
        init_populations_kernel<Real, Store, false><<<blocks_for(N), 256, 0, st>>>(rho, u, f, scale, N);
    return cudaGetLastError();
}

template <typename Store>
cudaError_t launch_decode_plane(const Store* f, double* dst, int N, const float* scale, cudaStream_t st)
{
    decode_plane_kernel<Store><<<blocks_for(N), 256, 0, st>>>(f, dst, N, scale);
    return cudaGetLastError();
}

template <typename Store>
cudaError_t launch_encode_plane(const double* src, Store* f, int N, const float* scale, cudaStream_t st)
{
    encode_plane_kernel<Store><<<blocks_for(N), 256, 0, st>>>(src, f, N, scale);
    return cudaGetLastError();
}

cudaError_t launch_scale_init(const float* rho, const float* u, const float* F, const double g[3], int N,
                              float* scales, unsigned* ctrl, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(ctrl, 0, 2 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    scale_probe_kernel<<<blocks_for(N), 256, 0, st>>>(rho, u, F, (float)g[0], (float)g[1], (float)g[2], N, ctrl);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    scale_set_kernel<<<1, 1, 0, st>>>(scales, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_trig_table(double* t, int nx, int ny, cudaStream_t st)
{
    trig_table_kernel<<<(nx + ny + 255) / 256, 256, 0, st>>>(t, nx, ny);
    return cudaGetLastError();
}

// The two-column kernel takes the plain path (no three-constant energy, no
// obstacles) when nx is even and every field pointer is aligned to its 2-vector
// (caller-owned buffers, as in the no-allocation entry point, may not be);
// otherwise the one-column kernel runs.
inline bool aligned_to(const void* p, size_t bytes) { return reinterpret_cast<uintptr_t>(p) % bytes == 0; }
inline bool diag_pairs(const DiagArgs& a)
{
    if (a.solid != nullptr || a.frank3 || a.g.nx % 2 != 0) return false;
    const size_t real2 = a.precision == NH_FP64 ? 16 : 8;
    const size_t store2 = a.precision == NH_FP64 ? 16 : (a.storage == NH_STORE_F32 ? 8 : 4);
    return aligned_to(a.f, store2) && aligned_to(a.n, real2) && aligned_to(a.u, real2) && aligned_to(a.rho, real2);
}

void launch_diag_pair_kernel(const DiagArgs& a, int blocks, cudaStream_t st)
{
    if (a.lbpart != nullptr) {  // the LB launch summed the populations, u and rho (F32 / F64 stores)
        if (a.precision == NH_FP64)
            diag_pair_kernel<double, double, true><<<blocks, DIAG_THREADS, 0, st>>>(a);
        else
            diag_pair_kernel<float, float, true><<<blocks, DIAG_THREADS, 0, st>>>(a);
        return;
    }
    if (a.precision == NH_FP64) {
        diag_pair_kernel<double, double><<<blocks, DIAG_THREADS, 0, st>>>(a);
        return;
    }
    switch (a.storage) {
    case NH_STORE_F32: diag_pair_kernel<float, float><<<blocks, DIAG_THREADS, 0, st>>>(a); break;
    case NH_STORE_F16S: diag_pair_kernel<float, __half><<<blocks, DIAG_THREADS, 0, st>>>(a); break;
    default: diag_pair_kernel<float, __nv_bfloat16><<<blocks, DIAG_THREADS, 0, st>>>(a); break;
    }
}

template <bool Solid>
void launch_diag_kernel(const DiagArgs& a, int blocks, cudaStream_t st)
{
    if (!Solid && a.lbpart != nullptr) {  // the LB launch summed the populations, u and rho (F32 / F64 stores)
        if (a.precision == NH_FP64) {
            if (a.frank3)
                diag_kernel<double, double, true, false, true><<<blocks, DIAG_THREADS, 0, st>>>(a);
            else
                diag_kernel<double, double, false, false, true><<<blocks, DIAG_THREADS, 0, st>>>(a);
        } else if (a.frank3) {
            diag_kernel<float, float, true, false, true><<<blocks, DIAG_THREADS, 0, st>>>(a);
        } else {
            diag_kernel<float, float, false, false, true><<<blocks, DIAG_THREADS, 0, st>>>(a);
        }
        return;
    }
    if (a.precision == NH_FP64) {
        if (a.frank3)
            diag_kernel<double, double, true, Solid><<<blocks, DIAG_THREADS, 0, st>>>(a);
        else
            diag_kernel<double, double, false, Solid><<<blocks, DIAG_THREADS, 0, st>>>(a);
    } else if (a.frank3) {
        switch (a.storage) {
        case NH_STORE_F32: diag_kernel<float, float, true, Solid><<<blocks, DIAG_THREADS, 0, st>>>(a); break;
        case NH_STORE_F16S: diag_kernel<float, __half, true, Solid><<<blocks, DIAG_THREADS, 0, st>>>(a); break;
        default: diag_kernel<float, __nv_bfloat16, true, Solid><<<blocks, DIAG_THREADS, 0, st>>>(a); break;
        }
    } else {
        switch (a.storage) {
        case NH_STORE_F32: diag_kernel<float, float, false, Solid><<<blocks, DIAG_THREADS, 0, st>>>(a); break;
        case NH_STORE_F16S: diag_kernel<float, __half, false, Solid><<<blocks, DIAG_THREADS, 0, st>>>(a); break;
        default: diag_kernel<float, __nv_bfloat16, false, Solid><<<blocks, DIAG_THREADS, 0, st>>>(a); break;
        }
    }
}

cudaError_t launch_diag_final(const double* partials, double* result, int blocks, int V, cudaStream_t st)
{
    diag_final_kernel<<<V, kFinalThreads, 0, st>>>(partials, result, blocks, V);
    return cudaGetLastError();
}

cudaError_t launch_diagnostics(const DiagArgs& a, cudaStream_t st)
{
    if (a.lbpart != nullptr && (a.solid != nullptr || (a.storage != NH_STORE_F32 && a.storage != NH_STORE_F64)))
        return cudaErrorInvalidValue;
    const bool pairs = diag_pairs(a);
    const bool nonly = a.lbpart != nullptr;  // the kernels read the director alone
    const int chunk = pairs ? (nonly ? kDiagPairChunkN : kDiagPairChunk) : (nonly ? kDiagChunkN : kDiagChunk);
    const int items = (pairs ? (a.g.nx / 2) : a.g.nx) * a.g.ny * ((a.g.nz + chunk - 1) / chunk);
    int blocks = (items + DIAG_THREADS - 1) / DIAG_THREADS;
    if (blocks > a.blocks) blocks = a.blocks;
    if (pairs && blocks > 4 * 152) blocks = 4 * 152;  // two-column kernel: 4 resident blocks on each of 152 SMs
    if (pairs)
        launch_diag_pair_kernel(a, blocks, st);
    else if (a.solid != nullptr)
        launch_diag_kernel<true>(a, blocks, st);
    else
        launch_diag_kernel<false>(a, blocks, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_final_kernel<<<diag_num_values(a.n_tubes), kFinalThreads, 0, st>>>(
        a.partials, a.result, blocks, diag_num_values(a.n_tubes));
    return cudaGetLastError();
}

template cudaError_t launch_load_fields<double>(const double*, const double*, const double*, double*, double*,
                                                double*, int, cudaStream_t);
template cudaError_t launch_load_fields<float>(const double*, const double*, const double*, float*, float*, float*,
                                               int, cudaStream_t);
template cudaError_t launch_store_vec<double>(const double*, double*, int64_t, cudaStream_t);
template cudaError_t launch_store_vec<float>(const float*, double*, int64_t, cudaStream_t);
template cudaError_t launch_init_populations<double, double>(const double*, const double*, double*, const float*,
                                                             int, bool, cudaStream_t);
template cudaError_t launch_init_populations<float, float>(const float*, const float*, float*, const float*, int,
                                                           bool, cudaStream_t);
template cudaError_t launch_init_populations<float, __half>(const float*, const float*, __half*, const float*, int,
                                                            bool, cudaStream_t);
template cudaError_t launch_init_populations<float, __nv_bfloat16>(const float*, const float*, __nv_bfloat16*,
                                                                   const float*, int, bool, cudaStream_t);
template cudaError_t launch_decode_plane<double>(const double*, double*, int, const float*, cudaStream_t);
template cudaError_t launch_decode_plane<float>(const float*, double*, int, const float*, cudaStream_t);
template cudaError_t launch_decode_plane<__half>(const __half*, double*, int, const float*, cudaStream_t);
template cudaError_t launch_decode_plane<__nv_bfloat16>(const __nv_bfloat16*, double*, int, const float*,
                                                        cudaStream_t);
template cudaError_t launch_encode_plane<double>(const double*, double*, int, const float*, cudaStream_t);
template cudaError_t launch_encode_plane<float>(const double*, float*, int, const float*, cudaStream_t);
template cudaError_t launch_encode_plane<__half>(const double*, __half*, int, const float*, cudaStream_t);
template cudaError_t launch_encode_plane<__nv_bfloat16>(const double*, __nv_bfloat16*, int, const float*,
                                                        cudaStream_t);

}  // namespace nh
