// fd.cu -- finite-difference director update and LC stress / force
// (arXiv:2503.06610, Secs. II.A-II.B, Eq. director-time-eq, Eq. force-lc-eq).
//
// Kernels (one thread per site, radius-1 stencils, central differences):
//   fd_predict : (dn/dt)_old from n and u;  n^P = n + dt_FD (dn/dt)_old
//   fd_correct : (dn/dt)_P from n^P and u;  n <- n + dt_FD/2 [(dn/dt)_old + (dn/dt)_P],
//                then n <- n/|n|  (in place: each site reads only its own n)
//   stress     : sigma = sigma^v(alpha_4') + sigma^e from the new n and u
//   force      : F_lc,a = d_b sigma_ab, zero stress at solid ghost layers
// The molecular field is the one-constant chiral form
//   h = K lap n - 2 K q0 curl n + W0 n_z z_hat
// (compact Laplacian, central curl).  Beyond the plates the ghost velocity is
// zero and the ghost director is z_hat (homeotropic) or the adjacent layer.
#include "nh_internal.cuh"

namespace nh {

namespace {

template <typename Real>
__device__ __forceinline__ void site_xyz(const Geom& g, int s, int& x, int& y, int& z)
{
    x = s % g.nx;
    const int t = s / g.nx;
    y = t % g.ny;
    z = t / g.ny;
}

// Director at (x, y, z) with x, y already wrapped; z may be -1 or nz.
template <typename Real>
__device__ __forceinline__ void dir_at(const Real* __restrict__ n, const Geom& g, int x, int y, int z, Real out[3])
{
    if (g.walls) {
        if (z < 0 || z >= g.nz) {
            if (g.anchoring == NH_ANCHOR_HOMEOTROPIC) {
                out[0] = Real(0);
                out[1] = Real(0);
                out[2] = Real(1);
                return;
            }
            z = z < 0 ? 0 : g.nz - 1;
        }
    } else {
        z = wrap_p(z, g.nz);
    }
    const int s = x + g.nx * (y + g.ny * z);
    out[0] = n[s];
    out[1] = n[g.N + s];
    out[2] = n[2 * g.N + s];
}

template <typename Real>
__device__ __forceinline__ void vel_at(const Real* __restrict__ u, const Geom& g, int x, int y, int z, Real out[3])
{
    if (g.walls) {
        if (z < 0 || z >= g.nz) {
            out[0] = out[1] = out[2] = Real(0);
            return;
        }
    } else {
        z = wrap_p(z, g.nz);
    }
    const int s = x + g.nx * (y + g.ny * z);
    out[0] = u[s];
    out[1] = u[g.N + s];
    out[2] = u[2 * g.N + s];
}

// 7-point neighbourhood: index 0 = centre, 1 + 2b = +e_b, 2 + 2b = -e_b.
template <typename Real>
__device__ __forceinline__ void gather7(const Real* __restrict__ f, const Geom& g, int x, int y, int z, Real v[7][3],
                                        bool director)
{
    const int xp = wrap_p(x + 1, g.nx), xm = wrap_p(x - 1, g.nx);
    const int yp = wrap_p(y + 1, g.ny), ym = wrap_p(y - 1, g.ny);
    if (director) {
        dir_at(f, g, x, y, z, v[0]);
        dir_at(f, g, xp, y, z, v[1]);
        dir_at(f, g, xm, y, z, v[2]);
        dir_at(f, g, x, yp, z, v[3]);
        dir_at(f, g, x, ym, z, v[4]);
        dir_at(f, g, x, y, z + 1, v[5]);
        dir_at(f, g, x, y, z - 1, v[6]);
    } else {
        vel_at(f, g, x, y, z, v[0]);
        vel_at(f, g, xp, y, z, v[1]);
        vel_at(f, g, xm, y, z, v[2]);
        vel_at(f, g, x, yp, z, v[3]);
        vel_at(f, g, x, ym, z, v[4]);
        vel_at(f, g, x, y, z + 1, v[5]);
        vel_at(f, g, x, y, z - 1, v[6]);
    }
}

// dn[b][c] = d_b n_c, du[a][m] = d_a u_m (central), molecular field h.
template <typename Real>
__device__ __forceinline__ void local_fields(const Real nn[7][3], const Real uu[7][3], const FDPar<Real>& p,
                                             Real dn[3][3], Real du[3][3], Real h[3])
{
    Real lap[3] = {0, 0, 0};
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            dn[b][c] = Real(0.5) * (nn[1 + 2 * b][c] - nn[2 + 2 * b][c]);
            du[b][c] = Real(0.5) * (uu[1 + 2 * b][c] - uu[2 + 2 * b][c]);
            lap[c] += nn[1 + 2 * b][c] + nn[2 + 2 * b][c] - Real(2) * nn[0][c];
        }
    const Real curl[3] = {dn[1][2] - dn[2][1], dn[2][0] - dn[0][2], dn[0][1] - dn[1][0]};
    const Real kq = Real(2) * p.K * p.q0;
#pragma unroll
    for (int a = 0; a < 3; ++a) h[a] = p.K * lap[a] - kq * curl[a];
    h[2] += p.W0 * nn[0][2];
}

// Eq. director-time-eq: dn_m/dt = h_m/g1 - (g2/g1) n_a D_am - u_g d_g n_m + W_mg n_g.
template <typename Real>
__device__ __forceinline__ void director_rate(const Real nn[7][3], const Real uu[7][3], const FDPar<Real>& p,
                                              Real rate[3])
{
    Real dn[3][3], du[3][3], h[3];
    local_fields(nn, uu, p, dn, du, h);
    const Real* n = nn[0];
    const Real* u = uu[0];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        Real r = h[m] * p.inv_gamma1;
        Real nD = 0, adv = 0, Wn = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            nD += n[a] * Real(0.5) * (du[a][m] + du[m][a]);   // n_a D_am
            adv += u[a] * dn[a][m];                            // u_g d_g n_m
            Wn += Real(0.5) * (du[a][m] - du[m][a]) * n[a];    // W_ma n_a, W_ma = (d_a u_m - d_m u_a)/2
        }
        rate[m] = r - p.g2_over_g1 * nD - adv + Wn;
    }
}

template <typename Real>
__device__ __forceinline__ void fd_predict_site(const FDChan<Real>& c, int s)
{
    int x, y, z;
    site_xyz<Real>(c.g, s, x, y, z);
    Real nn[7][3], uu[7][3], r[3];
    gather7(c.n, c.g, x, y, z, nn, true);
    gather7(c.u, c.g, x, y, z, uu, false);
    director_rate(nn, uu, c.p, r);
    const int N = c.g.N;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        c.ndot[a * N + s] = r[a];
        c.nP[a * N + s] = nn[0][a] + c.p.dt * r[a];
    }
}

template <typename Real>
__device__ __forceinline__ void fd_correct_site(const FDChan<Real>& c, int s)
{
    int x, y, z;
    site_xyz<Real>(c.g, s, x, y, z);
    Real nn[7][3], uu[7][3], r[3];
    gather7(c.nP, c.g, x, y, z, nn, true);
    gather7(c.u, c.g, x, y, z, uu, false);
    director_rate(nn, uu, c.p, r);
    const int N = c.g.N;
    Real nw[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) nw[a] = c.n[a * N + s] + c.p.dt * Real(0.5) * (c.ndot[a * N + s] + r[a]);
    const Real inv = Real(1) / sqrt(nw[0] * nw[0] + nw[1] * nw[1] + nw[2] * nw[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) c.n[a * N + s] = nw[a] * inv;
}

template <typename Real>
__device__ __forceinline__ void stress_site(const FDChan<Real>& c, int s)
{
    int x, y, z;
    site_xyz<Real>(c.g, s, x, y, z);
    Real nn[7][3], uu[7][3];
    gather7(c.n, c.g, x, y, z, nn, true);
    gather7(c.u, c.g, x, y, z, uu, false);
    Real dn[3][3], du[3][3], h[3];
    local_fields(nn, uu, c.p, dn, du, h);
    const Real* n = nn[0];
    const FDPar<Real>& p = c.p;
    Real D[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) D[a][b] = Real(0.5) * (du[a][b] + du[b][a]);
    Real Dn[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) Dn[a] = D[a][0] * n[0] + D[a][1] * n[1] + D[a][2] * n[2];
    const Real nDn = n[0] * Dn[0] + n[1] * Dn[1] + n[2] * Dn[2];
    const Real hn = h[0] * n[0] + h[1] * n[1] + h[2] * n[2];
    // kinematic transport from the director equation, projected normal to n
    Real Nv[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) Nv[m] = ((h[m] - hn * n[m]) - p.gamma2 * (Dn[m] - n[m] * nDn)) * p.inv_gamma1;
    // chi[b][g] = eps_{c b g} n_c
    const Real chi[3][3] = {{0, n[2], -n[1]}, {-n[2], 0, n[0]}, {n[1], -n[0], 0}};
    const int N = c.g.N;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            Real sv = p.a1 * n[a] * n[b] * nDn + p.a2 * n[b] * Nv[a] + p.a3 * n[a] * Nv[b] + p.a4p * D[a][b] +
                      p.a5 * n[b] * Dn[a] + p.a6 * n[a] * Dn[b];
            Real se = 0;
#pragma unroll
            for (int gg = 0; gg < 3; ++gg) se -= dn[a][gg] * (p.K * dn[b][gg] + p.K * p.q0 * chi[b][gg]);
            c.sigma[(3 * a + b) * N + s] = sv + se;
        }
}

template <typename Real>
__device__ __forceinline__ void force_site(const FDChan<Real>& c, int s)
{
    int x, y, z;
    site_xyz<Real>(c.g, s, x, y, z);
    const Geom& g = c.g;
    const int N = g.N;
    const int xp = wrap_p(x + 1, g.nx), xm = wrap_p(x - 1, g.nx);
    const int yp = wrap_p(y + 1, g.ny), ym = wrap_p(y - 1, g.ny);
    int zp = z + 1, zm = z - 1;
    bool zp_ok = true, zm_ok = true;
    if (g.walls) {
        zp_ok = zp < g.nz;
        zm_ok = zm >= 0;
    } else {
        zp = wrap_p(zp, g.nz);
        zm = wrap_p(zm, g.nz);
    }
    const int sxp = xp + g.nx * (y + g.ny * z), sxm = xm + g.nx * (y + g.ny * z);
    const int syp = x + g.nx * (yp + g.ny * z), sym = x + g.nx * (ym + g.ny * z);
    const int szp = x + g.nx * (y + g.ny * (zp_ok ? zp : 0)), szm = x + g.nx * (y + g.ny * (zm_ok ? zm : 0));
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const Real* sx = c.sigma + (3 * a + 0) * N;
        const Real* sy = c.sigma + (3 * a + 1) * N;
        const Real* sz = c.sigma + (3 * a + 2) * N;
        const Real dz = (zp_ok ? sz[szp] : Real(0)) - (zm_ok ? sz[szm] : Real(0));
        c.F[a * N + s] = Real(0.5) * ((sx[sxp] - sx[sxm]) + (sy[syp] - sy[sym]) + dz);
    }
}

template <typename Real, int Stage>
__device__ __forceinline__ void fd_stage_site(const FDChan<Real>& c, int s)
{
    if (Stage == 0)
        fd_predict_site(c, s);
    else if (Stage == 1)
        fd_correct_site(c, s);
    else if (Stage == 2)
        stress_site(c, s);
    else
        force_site(c, s);
}

template <typename Real, int Stage>
__global__ void __launch_bounds__(256) fd_kernel(const FDChan<Real> c)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < c.g.N) fd_stage_site<Real, Stage>(c, s);
}

// Batched FD stage: a persistent grid walks the (channel, tile) work list.
template <typename Real, int Stage>
__global__ void __launch_bounds__(256) fd_batch_kernel(const FDBatch<Real> b)
{
    const int total = b.prefix[b.count];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        int lo = 0, hi = b.count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (b.prefix[mid] <= t)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int s = (t - b.prefix[lo]) * blockDim.x + threadIdx.x;
        if (s < b.ch[lo].g.N) fd_stage_site<Real, Stage>(b.ch[lo], s);
    }
}

inline int blocks_for(int N) { return (N + 255) / 256; }

}  // namespace

template <typename Real>
cudaError_t launch_fd_batch(FDBatch<Real>& b, int stage, int grid, cudaStream_t st)
{
    if (b.count < 1 || b.count > kMaxBatch) return cudaErrorInvalidValue;
    b.prefix[0] = 0;
    for (int k = 0; k < b.count; ++k) b.prefix[k + 1] = b.prefix[k] + blocks_for(b.ch[k].g.N);
    const int blocks = grid < b.prefix[b.count] ? grid : b.prefix[b.count];
    switch (stage) {
    case 0: fd_batch_kernel<Real, 0><<<blocks, 256, 0, st>>>(b); break;
    case 1: fd_batch_kernel<Real, 1><<<blocks, 256, 0, st>>>(b); break;
    case 2: fd_batch_kernel<Real, 2><<<blocks, 256, 0, st>>>(b); break;
    default: fd_batch_kernel<Real, 3><<<blocks, 256, 0, st>>>(b); break;
    }
    return cudaGetLastError();
}
template cudaError_t launch_fd_batch<double>(FDBatch<double>&, int, int, cudaStream_t);
template cudaError_t launch_fd_batch<float>(FDBatch<float>&, int, int, cudaStream_t);

template <typename Real>
cudaError_t launch_fd_predict(const FDChan<Real>& c, cudaStream_t st)
{
    fd_kernel<Real, 0><<<blocks_for(c.g.N), 256, 0, st>>>(c);
    return cudaGetLastError();
}
template <typename Real>
cudaError_t launch_fd_correct(const FDChan<Real>& c, cudaStream_t st)
{
    fd_kernel<Real, 1><<<blocks_for(c.g.N), 256, 0, st>>>(c);
    return cudaGetLastError();
}
template <typename Real>
cudaError_t launch_stress(const FDChan<Real>& c, cudaStream_t st)
{
    fd_kernel<Real, 2><<<blocks_for(c.g.N), 256, 0, st>>>(c);
    return cudaGetLastError();
}
template <typename Real>
cudaError_t launch_force(const FDChan<Real>& c, cudaStream_t st)
{
    fd_kernel<Real, 3><<<blocks_for(c.g.N), 256, 0, st>>>(c);
    return cudaGetLastError();
}

template cudaError_t launch_fd_predict<double>(const FDChan<double>&, cudaStream_t);
template cudaError_t launch_fd_predict<float>(const FDChan<float>&, cudaStream_t);
template cudaError_t launch_fd_correct<double>(const FDChan<double>&, cudaStream_t);
template cudaError_t launch_fd_correct<float>(const FDChan<float>&, cudaStream_t);
template cudaError_t launch_stress<double>(const FDChan<double>&, cudaStream_t);
template cudaError_t launch_stress<float>(const FDChan<float>&, cudaStream_t);
template cudaError_t launch_force<double>(const FDChan<double>&, cudaStream_t);
template cudaError_t launch_force<float>(const FDChan<float>&, cudaStream_t);

}  // namespace nh
