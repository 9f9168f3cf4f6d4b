// lb.cu -- fused D3Q19 lattice-Boltzmann collide-and-stream sweep
// (arXiv:2503.06610, Sec. II.C).
//
// One thread owns SPT consecutive sites of an x-row (SPT = 2 when nx is even)
// and performs, in registers:
//   1. streaming by pull: f_i(x) <- f*_i(x - e_i) of the previous step, or the
//      half-way bounce-back f*_opp(i)(x) when x - e_i lies in a plate;
//   2. moments, Eqs. shifted-rho / shifeted-u (or the plain ones):
//      rho - 1 = sum_i f^s_i,  rho u = sum_i e_i f^s_i + F/2,  F = F_lc + rho g;
//   3. equilibrium (Eq. shifted-feq or Eq. feq-eq) and Guo source S_i^F;
//   4. SRT relaxation (Eq. shifted-lbe): f*_i = f_i - (f_i - f^eq_i)/tau
//      + (1 - 1/(2 tau)) S_i^F, written to the other population buffer.
// Populations are structure-of-arrays planes [19][N]: every warp reads and
// writes 19 runs of consecutive sites, coalesced.  Planes with e_x = 0 are
// read and all planes written as aligned 2-site vectors; the +-1 x shift of
// the other planes is served from L1/L2.  The relaxation uses the symmetry of
// each pair (e_i, -e_i): the parts of f^eq and S_i that are even in e_i are
// computed once per pair and the odd parts change sign.  u and rho are written
// only on steps that feed an FD update (or end a call); such a launch can also
// leave per-block partial sums for the diagnostics (mass, max |u|, non-finite
// count), so that the diagnostics of that state need not read the
// populations, u and rho again.
#include <type_traits>

#include "nh_internal.cuh"

#include <string.h>

namespace nh {

constexpr int kLBThreads = 256;

// Power-of-two scale that puts m near 2^kScaleHeadroomLog2 (exact in float).
__device__ __forceinline__ float scale_for(float m, float fallback)
{
    if (!(m > 0.f) || !isfinite(m)) return fallback;
    int e;
    frexpf(m, &e);  // m < 2^e
    int k = kScaleHeadroomLog2 - e;
    k = k < -120 ? -120 : (k > 120 ? 120 : k);
    return ldexpf(1.f, k);
}

template <typename Store>
struct Vec2;
template <>
struct Vec2<double> {
    using T = double2;
};
template <>
struct Vec2<float> {
    using T = float2;
};
template <>
struct Vec2<__half> {
    using T = __half2;
};
template <>
struct Vec2<__nv_bfloat16> {
    using T = __nv_bfloat162;
};

template <typename Store, typename Real>
__device__ __forceinline__ void load2(const Store* p, float inv, Real& a, Real& b)
{
    const typename Vec2<Store>::T v = *reinterpret_cast<const typename Vec2<Store>::T*>(p);
    if constexpr (std::is_same<Store, __half>::value) {
        const float2 fv = __half22float2(v);
        a = fv.x * inv;
        b = fv.y * inv;
    } else if constexpr (std::is_same<Store, __nv_bfloat16>::value) {
        const float2 fv = __bfloat1622float2(v);
        a = fv.x * inv;
        b = fv.y * inv;
    } else {
        a = v.x;
        b = v.y;
    }
}

template <typename Store, typename Real>
__device__ __forceinline__ void store2(Store* p, Real a, Real b, float scale)
{
    typename Vec2<Store>::T v;
    if constexpr (std::is_same<Store, __half>::value) {
        v = __floats2half2_rn(a * scale, b * scale);
    } else if constexpr (std::is_same<Store, __nv_bfloat16>::value) {
        v = __floats2bfloat162_rn(a * scale, b * scale);
    } else {
        v.x = a;
        v.y = b;
    }
    *reinterpret_cast<typename Vec2<Store>::T*>(p) = v;
}

// Four consecutive sites (16-byte aligned for FP32, 8-byte for the 16-bit stores).
template <typename Store>
__device__ __forceinline__ float2 vec2_to_float2(typename Vec2<Store>::T v)
{
    if constexpr (std::is_same<Store, __half>::value)
        return __half22float2(v);
    else
        return __bfloat1622float2(v);
}

template <typename Store, typename Real>
__device__ __forceinline__ void load4(const Store* p, float inv, Real v[4])
{
    if constexpr (sizeof(Store) == 2) {
        using V2 = typename Vec2<Store>::T;
        const uint2 raw = *reinterpret_cast<const uint2*>(p);
        V2 lo, hi;
        memcpy(&lo, &raw.x, 4);
        memcpy(&hi, &raw.y, 4);
        const float2 a = vec2_to_float2<Store>(lo), b = vec2_to_float2<Store>(hi);
        v[0] = a.x * inv;
        v[1] = a.y * inv;
        v[2] = b.x * inv;
        v[3] = b.y * inv;
    } else if constexpr (std::is_same<Store, float>::value) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
    } else {
        const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
        v[0] = a.x;
        v[1] = a.y;
        v[2] = b.x;
        v[3] = b.y;
    }
}

template <typename Store, typename Real>
__device__ __forceinline__ void store4(Store* p, const Real v[4], float scale)
{
    if constexpr (std::is_same<Store, __half>::value || std::is_same<Store, __nv_bfloat16>::value) {
        using V2 = typename Vec2<Store>::T;
        V2 lo, hi;
        if constexpr (std::is_same<Store, __half>::value) {
            lo = __floats2half2_rn(v[0] * scale, v[1] * scale);
            hi = __floats2half2_rn(v[2] * scale, v[3] * scale);
        } else {
            lo = __floats2bfloat162_rn(v[0] * scale, v[1] * scale);
            hi = __floats2bfloat162_rn(v[2] * scale, v[3] * scale);
        }
        uint2 raw;
        memcpy(&raw.x, &lo, 4);
        memcpy(&raw.y, &hi, 4);
        *reinterpret_cast<uint2*>(p) = raw;
    } else if constexpr (std::is_same<Store, float>::value) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
    }
}

// Scale controller, barrier form: the block's warps combine their maxima
// (amax already reduced over each warp, in population units) in wmax, one
// thread folds the block maximum into the launch's running maximum c.ctrl[0]
// and takes a ticket c.ctrl[1]; the launch's last block records the scale of
// the buffer just written and sets the target of the next step.
template <typename Real, typename Store>
__device__ __forceinline__ void scale_controller_block(const LBChan<Real, Store>& c, float amax, float scale_out,
                                                       int ntiles, float* wmax, bool& last)
{
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = amax;
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = fmaxf(b, wmax[w]);
        if (b > __int_as_float((int)__ldcg(&c.ctrl[0])))
            atomicMax(reinterpret_cast<int*>(&c.ctrl[0]), __float_as_int(b));
        __threadfence();
        const unsigned ticket = atomicAdd(&c.ctrl[1], 1u);
        last = ticket == (unsigned)ntiles - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const float m = __int_as_float((int)atomicExch(&c.ctrl[0], 0u));
        c.scales[1 - c.src] = scale_out;
        c.scales[2] = scale_for(m, scale_out);
        c.ctrl[1] = 0u;
    }
    __syncthreads();  // the shared controller state is reused by the next tile
}

// Rounded products and fused multiply-adds written out: the compiler may not
// contract a*b + c on its own here, so every launch shape and kernel that
// collides a site (single channels, batches, the row-staged kernel) rounds
// in the same order and gives the same bits.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return fma(a, b, c); }

// e . v for a lattice vector with components in {-1, 0, 1} (constants once the
// direction loop is unrolled): sums and differences only.
template <typename Real>
__device__ __forceinline__ Real edot(int X, int Y, int Z, Real vx, Real vy, Real vz)
{
    Real r = Real(0);
    if (X != 0) r = X > 0 ? vx : -vx;
    if (Y != 0) r = (X != 0) ? (Y > 0 ? r + vy : r - vy) : (Y > 0 ? vy : -vy);
    if (Z != 0) r = (X != 0 || Y != 0) ? (Z > 0 ? r + vz : r - vz) : (Z > 0 ? vz : -vz);
    return r;
}

// Moments, equilibrium, Guo source and relaxation of one site s from its
// streamed populations f (decoded values; raw 2^k-scaled ones for the 16-bit
// stores, whose power-of-two factors inv_in and scale_out are folded in) and
// its liquid-crystal force F_lc = (flx, fly, flz) (the body force rho g is added here), into
// fo; u and rho written when Macro >= 1, the diagnostics partials accumulated
// when Macro == 2, the largest |fo| (encoded units) into amax for the 16-bit
// scale controller.  Every launch shape calls this for every site, and its
// rounding order is explicit, so all shapes give bit-identical results.
template <typename Real, typename Store, bool Shifted, int Macro>
__device__ __forceinline__ void lb_collide_site(const LBChan<Real, Store>& c, int s, const Real (&f)[19],
                                                Real (&fo)[19], Real flx, Real fly, Real flz, float inv_in,
                                                float scale_out, Real& psum, Real& pmax, int& pbad, float& amax)
{
    NH_D3Q19_TABLES
    constexpr bool kScaled = sizeof(Store) == 2;
    constexpr bool WriteMacro = Macro >= 1;
    constexpr bool Partials = Macro == 2;
    const int N = c.g.N;
    // 2. moments: pair sums and differences of (e_i, -e_i)
    Real sum = f[0], mx = 0, my = 0, mz = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int i = 2 * k + 1;
        sum += f[i] + f[i + 1];
        const Real d = f[i] - f[i + 1];
        if (EX[i] != 0) mx += EX[i] > 0 ? d : -d;
        if (EY[i] != 0) my += EY[i] > 0 ? d : -d;
        if (EZ[i] != 0) mz += EZ[i] > 0 ? d : -d;
    }
    if (kScaled) {  // raw populations: scale the sums once
        sum = mul_rn(sum, Real(inv_in));
        mx = mul_rn(mx, Real(inv_in));
        my = mul_rn(my, Real(inv_in));
        mz = mul_rn(mz, Real(inv_in));
    }
    const Real rho = Shifted ? Real(1) + sum : sum;
    const Real drho = Shifted ? sum : sum - Real(1);
    const Real Fx = fma_rn(rho, c.gx, flx);
    const Real Fy = fma_rn(rho, c.gy, fly);
    const Real Fz = fma_rn(rho, c.gz, flz);
    const Real inv_rho = Real(1) / rho;
    Real Hx = Fx, Hy = Fy, Hz = Fz;  // force whose half shifts u
    if (c.Fu != nullptr) {
        Hx = fma_rn(rho, c.gx, c.Fu[s]);
        Hy = fma_rn(rho, c.gy, c.Fu[N + s]);
        Hz = fma_rn(rho, c.gz, c.Fu[2 * N + s]);
    }
    const Real ux = mul_rn(fma_rn(Real(0.5), Hx, mx), inv_rho);
    const Real uy = mul_rn(fma_rn(Real(0.5), Hy, my), inv_rho);
    const Real uz = mul_rn(fma_rn(Real(0.5), Hz, mz), inv_rho);
    if (WriteMacro) {
        c.u[s] = ux;
        c.u[N + s] = uy;
        c.u[2 * N + s] = uz;
        c.rho[s] = rho;
    }

    // 3-4. equilibrium, Guo source and relaxation, per (e_i, -e_i) pair:
    //   f^eq = w rho [3 eu + 4.5 eu^2 - 1.5 u.u] + w (rho - 1 | rho)
    //   S    = w [3 eF + 9 eu eF - 3 u.F]
    //   f*   = (1 - omega) f + omega f^eq + (1 - omega/2) S
    // with a 16-bit store the constants carry scale_out (and omc the raw
    // input's inv_in), so fo[] leaves here already in encoded units
    const Real so = kScaled ? Real(scale_out) : Real(1);
    const Real omega = mul_rn(c.omega, so);
    const Real omc = mul_rn(Real(1) - c.omega, kScaled ? mul_rn(Real(inv_in), so) : Real(1));
    const Real cS = mul_rn(fma_rn(Real(-0.5), c.omega, Real(1)), so);
    const Real u2 = fma_rn(uz, uz, fma_rn(uy, uy, mul_rn(ux, ux)));
    const Real uu15 = mul_rn(Real(1.5), u2);
    const Real uF3 = mul_rn(Real(3), fma_rn(uz, Fz, fma_rn(uy, Fy, mul_rn(ux, Fx))));
    const Real base = Shifted ? drho : rho;
    // rest population (w = 1/3)
    {
        const Real w = Real(1) / Real(3);
        const Real t = fma_rn(-rho, uu15, base);
        fo[0] = fma_rn(omc, f[0], fma_rn(mul_rn(omega, w), t, -mul_rn(mul_rn(cS, w), uF3)));
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int i = 2 * k + 1;
        const Real w = i < 7 ? Real(1) / Real(18) : Real(1) / Real(36);
        const Real ow = mul_rn(omega, w);
        const Real A = mul_rn(ow, rho);
        const Real B = mul_rn(ow, base);
        const Real C = mul_rn(cS, w);
        const Real eu = edot(EX[i], EY[i], EZ[i], ux, uy, uz);
        const Real eF = edot(EX[i], EY[i], EZ[i], Fx, Fy, Fz);
        const Real X = fma_rn(mul_rn(Real(4.5), eu), eu, -uu15);
        const Real Y = fma_rn(mul_rn(Real(9), eu), eF, -uF3);
        const Real even = fma_rn(C, Y, fma_rn(A, X, B));
        const Real odd = mul_rn(Real(3), fma_rn(A, eu, mul_rn(C, eF)));
        fo[i] = fma_rn(omc, f[i], even) + odd;
        fo[i + 1] = fma_rn(omc, f[i + 1], even) - odd;
    }
    if (Partials) {  // the sums nh_diagnostics forms from the stored state, site by site
        Real fs = fo[0];
#pragma unroll
        for (int i = 1; i < 19; ++i) fs += fo[i];
        psum += fs;
        // max |u|^2 here and one square root per warp: sqrt is monotonic and
        // correctly rounded, so this equals the maximum of the per-site |u|
        pmax = max(pmax, u2);
        if (!isfinite(u2) || !isfinite(rho) || !isfinite(fs)) pbad += 1;
    }
    if (kScaled) {
#pragma unroll
        for (int i = 0; i < 19; ++i) amax = fmaxf(amax, fabsf((float)fo[i]));
    }
}

// Macro: 0 = populations only; 1 = also u and rho; 2 = also the diagnostics'
// block partials c.part[k * ntiles + tile] of k = 0: sum of the stored
// post-collision populations, 1: max |u|, 2: sites with a non-finite u, rho
// or population sum (FP32 and FP64 stores).
// One tile (one thread block's worth of sites) of one channel.  `tile` is the
// tile index within the channel and `ntiles` the channel's tile count (used by
// the 16-bit scale controller to find the channel's last tile).  Solid: the
// channel has obstacles (c.solid): a link whose source is a solid node
// bounces back half-way like the plates, and a solid node carries its
// populations over unchanged (u = 0, rho = 1 on macro steps); one site per thread.
// OneTile: the block sweeps this one tile (lb_kernel); the 16-bit scale
// controller then combines the warps through shared-memory atomics, and the
// block's last warp to finish carries the block's maximum on, so no warp waits
// at a barrier for the others.  A block of the batched kernel sweeps several
// tiles and keeps the barrier form.
template <typename Real, typename Store, bool Shifted, int Macro, int SPT, bool Solid = false, bool OneTile = false>
__device__ __forceinline__ void lb_tile(const LBChan<Real, Store>& c, int tile, int ntiles)
{
    static_assert(!Solid || SPT == 1, "obstacles use one site per thread");
    NH_D3Q19_TABLES
    constexpr bool kScaled = sizeof(Store) == 2;
    constexpr bool WriteMacro = Macro >= 1;
    constexpr bool Partials = Macro == 2;
    static_assert(!Partials || (!kScaled && !Solid), "diagnostics partials: FP32 / FP64 stores without obstacles");
    Real psum = 0, pmax = 0;  // diagnostics partials of this thread (Partials)
    int pbad = 0;
    __shared__ unsigned blk_max, blk_done;  // OneTile scale controller: block max (float bits), warps done
    if constexpr (kScaled && OneTile) {
        if (threadIdx.x == 0) {
            blk_max = 0u;
            blk_done = 0u;
        }
        __syncthreads();
    }
    const int N = c.g.N;
    const int s0 = (tile * blockDim.x + threadIdx.x) * SPT;
    float amax = 0.f;
    float scale_out = 1.f;
    if (kScaled) scale_out = c.scales[2];
    if (s0 < N) {
        const int nx = c.g.nx, ny = c.g.ny, nz = c.g.nz;
        const int x0 = s0 % nx;
        const int r = s0 / nx;
        const int y = r % ny;
        const int z = r / ny;
        const float inv_in = kScaled ? 1.f / c.scales[c.src] : 1.f;
        // 16-bit stores: the populations are read raw (still scaled by 2^k) and
        // the power-of-two factors inv_in and scale_out are folded into the
        // moments and the collision constants below; products with powers of two
        // are exact, so the results equal decoding, colliding and re-encoding
        const float ld = 1.f;
        const int plane_xy = nx * ny;

        // site deltas of the pull sources x - e (periodic in x and y; in z
        // periodic or replaced by bounce-back at the plates)
        int dxm[SPT], dxp[SPT];  // source x-1 (e_x = +1), x+1 (e_x = -1)
#pragma unroll
        for (int j = 0; j < SPT; ++j) {
            const int x = x0 + j;
            dxm[j] = x == 0 ? nx - 1 : -1;
            dxp[j] = x == nx - 1 ? -(nx - 1) : 1;
        }
        const int dym = (y == 0 ? ny - 1 : -1) * nx;
        const int dyp = (y == ny - 1 ? -(ny - 1) : 1) * nx;
        const int dzm = (z == 0 ? nz - 1 : -1) * plane_xy;
        const int dzp = (z == nz - 1 ? -(nz - 1) : 1) * plane_xy;
        const bool bb_lo = c.g.walls && z == 0;
        const bool bb_hi = c.g.walls && z == nz - 1;
        // the Solid variant also serves channels without a mask in a batch that has obstacles
        const bool solid_here = Solid && c.solid != nullptr && c.solid[s0] != 0;

        // 1. pull streaming with half-way bounce-back
        Real f[SPT][19];
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const bool bb = (EZ[i] > 0 && bb_lo) || (EZ[i] < 0 && bb_hi);
            const int row = (EY[i] > 0 ? dym : (EY[i] < 0 ? dyp : 0)) + (EZ[i] > 0 ? dzm : (EZ[i] < 0 ? dzp : 0));
            if (Solid) {
                const int dx = EX[i] > 0 ? dxm[0] : (EX[i] < 0 ? dxp[0] : 0);
                const int src = s0 + row + dx;
                const bool back = bb || (!solid_here && c.solid != nullptr && c.solid[src] != 0);
                const int k = back ? OPP[i] : i;
                f[0][i] = Codec<Store, Real>::load(c.fsrc + (size_t)(solid_here ? i : k) * N +
                                                       (solid_here || back ? s0 : src),
                                                   ld);
                continue;
            }
            const Store* plane = c.fsrc + (size_t)(bb ? OPP[i] : i) * N;
            if constexpr (SPT == 4) {
                // four sites of a row (nx % 4 == 0): aligned 4-site chunks of the
                // source row; e_x = +-1 reads two chunks and selects
                Real a[4];
                if (EX[i] == 0 || bb) {
                    load4(plane + (bb ? s0 : s0 + row), ld, a);
#pragma unroll
                    for (int j = 0; j < 4; ++j) f[j][i] = a[j];
                } else {
                    const Store* src = plane + s0 + row;  // chunk x0 .. x0 + 3 of the source row
                    Real b[4];
                    load4(src, ld, a);
                    if (EX[i] > 0) {  // sources x0 - 1 .. x0 + 2
                        load4(src + (x0 == 0 ? nx - 4 : -4), ld, b);
                        f[0][i] = b[3];
                        f[1][i] = a[0];
                        f[2][i] = a[1];
                        f[3][i] = a[2];
                    } else {  // sources x0 + 1 .. x0 + 4
                        load4(src + (x0 + 4 == nx ? -(nx - 4) : 4), ld, b);
                        f[0][i] = a[1];
                        f[1][i] = a[2];
                        f[2][i] = a[3];
                        f[3][i] = b[0];
                    }
                }
                continue;
            }
            if (SPT == 2 && EX[i] == 0) {
                load2(plane + (bb ? s0 : s0 + row), ld, f[0][i], f[SPT - 1][i]);
            } else {
#pragma unroll
                for (int j = 0; j < SPT; ++j) {
                    const int dx = EX[i] > 0 ? dxm[j] : (EX[i] < 0 ? dxp[j] : 0);
                    f[j][i] = Codec<Store, Real>::load(plane + (bb ? s0 + j : s0 + j + row + dx), ld);
                }
            }
        }

        Real fo[SPT][19];
        if (solid_here) {
#pragma unroll
            for (int i = 0; i < 19; ++i) fo[0][i] = kScaled ? f[0][i] * Real(inv_in * scale_out) : f[0][i];
            if (WriteMacro) {
                c.u[s0] = Real(0);
                c.u[N + s0] = Real(0);
                c.u[2 * N + s0] = Real(0);
                c.rho[s0] = Real(1);
            }
        }
#pragma unroll
        for (int j = 0; j < SPT; ++j) {
            if (solid_here) break;
            const int s = s0 + j;
            lb_collide_site<Real, Store, Shifted, Macro>(c, s, f[j], fo[j], c.F[s], c.F[N + s], c.F[2 * N + s], inv_in,
                                                        scale_out, psum, pmax, pbad, amax);
        }
        if (kScaled) amax /= scale_out;  // back to population units for the controller

        // store (aligned 2-site vectors when SPT = 2)
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            Store* dst = c.fdst + (size_t)i * N + s0;
            if constexpr (SPT == 4) {
                const Real v[4] = {fo[0][i], fo[1][i], fo[2][i], fo[3][i]};
                store4(dst, v, kScaled ? 1.f : scale_out);
            } else if (SPT == 2) {
                store2(dst, fo[0][i], fo[SPT - 1][i], kScaled ? 1.f : scale_out);
            } else {
                Codec<Store, Real>::store(dst, fo[0][i], kScaled ? 1.f : scale_out);
            }
        }
    }
    if constexpr (Partials) {
        // block partials: warp sums in the build's precision (FP64 arithmetic is
        // scarce on GB300: a per-thread FP64 reduction would cost a third of the
        // launch), then FP64 across the block's warps in a fixed order
        __shared__ double pred[kLBThreads / 32][3];
        Real m = psum, mx = pmax;
        for (int o = 16; o > 0; o >>= 1) {
            m += __shfl_xor_sync(0xffffffffu, m, o);
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        const int nb = __reduce_add_sync(0xffffffffu, pbad);
        if ((threadIdx.x & 31) == 0) {
            pred[threadIdx.x >> 5][0] = (double)m;
            pred[threadIdx.x >> 5][1] = (double)sqrt(mx);
            pred[threadIdx.x >> 5][2] = (double)nb;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double v[3] = {0.0, 0.0, 0.0};
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                v[0] += pred[w][0];
                v[1] = fmax(v[1], pred[w][1]);
                v[2] += pred[w][2];
            }
            for (int k = 0; k < 3; ++k) c.part[(size_t)k * ntiles + tile] = v[k];
        }
    }
    if (kScaled) {
        // In-kernel scale controller: block max -> global running max; the last
        // block to finish records the scale of the buffer just written and sets
        // the target of the next step from this step's max |f*|.
        __shared__ float wmax[kLBThreads / 32];
        __shared__ bool last;
        for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        if constexpr (OneTile) {
            if ((threadIdx.x & 31) == 0) {
                atomicMax(&blk_max, __float_as_uint(amax));  // amax >= 0: the bits order as the values
                __threadfence_block();
                if (atomicAdd(&blk_done, 1u) == (blockDim.x >> 5) - 1) {  // the block's last warp
                    __threadfence_block();
                    const float b = __uint_as_float(atomicAdd(&blk_max, 0u));
                    if (b > __int_as_float((int)__ldcg(&c.ctrl[0])))
                        atomicMax(reinterpret_cast<int*>(&c.ctrl[0]), __float_as_int(b));
                    __threadfence();
                    if (atomicAdd(&c.ctrl[1], 1u) == (unsigned)ntiles - 1) {  // the launch's last block
                        __threadfence();
                        const float m = __int_as_float((int)atomicExch(&c.ctrl[0], 0u));
                        c.scales[1 - c.src] = scale_out;
                        c.scales[2] = scale_for(m, scale_out);
                        c.ctrl[1] = 0u;
                    }
                }
            }
            return;
        }
        scale_controller_block(c, amax, scale_out, ntiles, wmax, last);
    }
}

template <typename Real, typename Store, bool Shifted, int Macro, int SPT, bool Solid = false>
__global__ void __launch_bounds__(kLBThreads) lb_kernel(const LBChan<Real, Store> c)
{
    lb_tile<Real, Store, Shifted, Macro, SPT, Solid, true>(c, blockIdx.x, gridDim.x);
}

// ------------------------------------------------------------------ 16-bit stores: rows staged by bulk copies
//
// The 16-bit kernels above are bound by latency and issue, not by HBM: each
// thread must hold its sites' 19 populations in registers while the loads are
// in flight, so the bytes in flight per SM are capped by the register file.
// lb_rows_kernel moves the streaming step to the copy engine.  A persistent
// block walks the x-rows (y, z) of the lattice; the row needs, per direction
// i, source row (y - e_y, z - e_z) of plane i, or its own row of plane opp(i)
// where e_i crosses a plate (half-way bounce-back): nx contiguous 16-bit
// values that one cp.async.bulk copies whole into shared memory, completing on
// the stage's mbarrier, together with the row's three force rows F_lc (the
// other load of the collision, which would otherwise wait on HBM latency).  kRowStages stages keep the copies of the next row in
// flight while the block collides the current one; the e_x = +-1 shift and the
// periodic x wrap are resolved by indexing the staged row.  Thread t owns the
// kRowSPT sites x = 4t .. 4t + 3 of the row (blockDim.x = nx / 4), read as
// aligned 4-site chunks as in the four-site register shape, and collides them
// with lb_collide_site, the code of every other shape, so the results are
// bit-identical to theirs.  Requirements (checked by lb_rows_valid): 16-bit
// stores, nx a multiple of 128 (whole warps; 16-byte aligned rows and planes)
// and at most kRowMaxNx, no obstacles.  Every mbarrier wait is bounded: on
// expiry the block records the timeout in c.ctrl[2], stops sweeping, waits
// (bounded) for the copies it issued and still takes its controller ticket.
constexpr int kRowSPT = 4;        // sites per thread: four consecutive sites of the row
constexpr int kRowStages = 2;      // rows in shared memory per block: the one collided, the next in flight
constexpr int kRowMaxNx = 256;
constexpr int kRowMinBlocks = 8;   // per SM: at most 128 registers a thread (64 threads at nx = 256)

namespace {

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool row_bar_wait(uint32_t bar, uint32_t parity)
{
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Direction of lane i < 19 of the issuing warp, packed in one register:
// (e_y + 1) | (e_z + 1) << 2 | opp(i) << 4.
__device__ __forceinline__ int row_lane(int lane)
{
    NH_D3Q19_TABLES
    int d = 0;
#pragma unroll
    for (int i = 0; i < 19; ++i)
        if (lane == i) d = (EY[i] + 1) | ((EZ[i] + 1) << 2) | (OPP[i] << 4);
    return d;
}

// Warp 0: the source rows of row r into one stage, completing on bar.  Lane
// 0 arms the barrier with the stage's bytes, then lane i < 19 copies
// direction i -- row (y - e_y, z - e_z) of plane i, or its own row of plane
// opp(i) where e_i crosses a plate -- to dst, and lanes 19 .. 21 copy row r of
// the three components of the force F_lc to fdst.
template <typename Store, typename Real>
__device__ __forceinline__ void issue_row(const Store* fsrc, const Real* F, const Geom& g, int r, Store* dst,
                                          Real* fdst, uint32_t bar)
{
    const uint32_t row_bytes = (uint32_t)g.nx * sizeof(Store);
    const uint32_t force_bytes = (uint32_t)g.nx * sizeof(Real);
    const int lane = (int)threadIdx.x & 31;
    if (lane == 0)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar),
                     "r"(19u * row_bytes + 3u * force_bytes)
                     : "memory");
    __syncwarp();
    if (lane < 19) {
        const int y = r % g.ny, z = r / g.ny;
        const int d = row_lane(lane);
        const int ey = (d & 3) - 1, ez = ((d >> 2) & 3) - 1, opp = d >> 4;
        const bool bb = g.walls && ((ez > 0 && z == 0) || (ez < 0 && z == g.nz - 1));
        const Store* src;
        if (bb) {
            src = fsrc + (size_t)opp * g.N + (size_t)r * g.nx;
        } else {
            int ys = y - ey, zs = z - ez;
            ys = ys < 0 ? ys + g.ny : (ys >= g.ny ? ys - g.ny : ys);
            zs = zs < 0 ? zs + g.nz : (zs >= g.nz ? zs - g.nz : zs);
            src = fsrc + (size_t)lane * g.N + (size_t)(ys + g.ny * zs) * g.nx;
        }
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                smem_addr(dst + (size_t)lane * g.nx)),
            "l"(src), "r"(row_bytes), "r"(bar)
            : "memory");
    } else if (lane < 22) {
        const int a = lane - 19;
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                smem_addr(fdst + (size_t)a * g.nx)),
            "l"(F + (size_t)a * g.N + (size_t)r * g.nx), "r"(force_bytes), "r"(bar)
            : "memory");
    }
}

}  // namespace

template <typename Real, typename Store, bool Shifted, int Macro>
__global__ void __launch_bounds__(kRowMaxNx / kRowSPT, kRowMinBlocks) lb_rows_kernel(const LBChan<Real, Store> c)
{
    static_assert(sizeof(Store) == 2 && Macro < 2, "row staging: 16-bit stores, no diagnostics partials");
    static_assert(kRowSPT == 4, "the staged rows are read as aligned 4-site chunks");
    static_assert(std::is_same<Real, float>::value, "16-bit stores compute in FP32");
    NH_D3Q19_TABLES
    extern __shared__ __align__(128) unsigned char rows_smem[];
    __shared__ __align__(8) uint64_t full[kRowStages];
    __shared__ float wmax[kRowMaxNx / kRowSPT / 32];
    __shared__ bool last;
    const Geom& g = c.g;
    const int nx = g.nx, N = g.N;
    // stage q: 19 population rows (Store) then the 3 force rows (Real) of one x-row
    const size_t pop_bytes = (size_t)19 * nx * sizeof(Store);
    const size_t stage_bytes = pop_bytes + (size_t)3 * nx * sizeof(Real);
    auto pop_stage = [&](int q) { return reinterpret_cast<Store*>(rows_smem + (size_t)q * stage_bytes); };
    auto force_stage = [&](int q) { return reinterpret_cast<Real*>(rows_smem + (size_t)q * stage_bytes + pop_bytes); };
    const int rows = g.ny * g.nz;
    const int my_rows = (int)blockIdx.x < rows ? (rows - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const float inv_in = 1.f / c.scales[c.src];
    const float scale_out = c.scales[2];
    const int x0 = kRowSPT * (int)threadIdx.x;
    Real psum = 0, pmax = 0;  // unused: no partials with 16-bit stores
    int pbad = 0;
    float amax = 0.f;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < kRowStages; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&full[k])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    const bool issuer = threadIdx.x < 32;  // warp 0 issues the copies, one direction per lane
    if (issuer)
        for (int k = 0; k < kRowStages && k < my_rows; ++k)
            issue_row(c.fsrc, c.F, g, (int)blockIdx.x + k * (int)gridDim.x, pop_stage(k), force_stage(k),
                      smem_addr(&full[k]));
    int k = 0;
    bool timed_out = false;
    for (; k < my_rows; ++k) {
        const int stage = k % kRowStages;
        const bool ok = row_bar_wait(smem_addr(&full[stage]), (uint32_t)(k / kRowStages) & 1u);
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        const int r = (int)blockIdx.x + k * (int)gridDim.x;
        const Store* st = pop_stage(stage);
        const int z = r / g.ny;
        Real f[kRowSPT][19];
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const bool bb = g.walls && ((EZ[i] > 0 && z == 0) || (EZ[i] < 0 && z == g.nz - 1));
            const Store* row = st + (size_t)i * nx;
            // aligned 4-site chunks of the staged row; e_x = +-1 takes one value of the neighbouring chunk
            Real a[4];
            load4(row + x0, 1.f, a);
            if (EX[i] == 0 || bb) {
#pragma unroll
                for (int j = 0; j < 4; ++j) f[j][i] = a[j];
            } else if (EX[i] > 0) {  // sources x0 - 1 .. x0 + 2
                Real b[4];
                load4(row + (x0 == 0 ? nx - 4 : x0 - 4), 1.f, b);
                f[0][i] = b[3];
                f[1][i] = a[0];
                f[2][i] = a[1];
                f[3][i] = a[2];
            } else {  // sources x0 + 1 .. x0 + 4
                Real b[4];
                load4(row + (x0 + 4 == nx ? 0 : x0 + 4), 1.f, b);
                f[0][i] = a[1];
                f[1][i] = a[2];
                f[2][i] = a[3];
                f[3][i] = b[0];
            }
        }
        float4 fl[3];  // F_lc of the thread's four sites, per component
#pragma unroll
        for (int a = 0; a < 3; ++a) fl[a] = *reinterpret_cast<const float4*>(force_stage(stage) + a * nx + x0);
        __syncthreads();  // the stage is read: refill it with the row kRowStages ahead
        if (issuer && k + kRowStages < my_rows)
            issue_row(c.fsrc, c.F, g, (int)blockIdx.x + (k + kRowStages) * (int)gridDim.x, pop_stage(stage),
                      force_stage(stage), smem_addr(&full[stage]));
        const int s0 = r * nx + x0;
        Real fo[kRowSPT][19];
#pragma unroll
        for (int j = 0; j < kRowSPT; ++j) {
            const float fx = j == 0 ? fl[0].x : (j == 1 ? fl[0].y : (j == 2 ? fl[0].z : fl[0].w));
            const float fy = j == 0 ? fl[1].x : (j == 1 ? fl[1].y : (j == 2 ? fl[1].z : fl[1].w));
            const float fz = j == 0 ? fl[2].x : (j == 1 ? fl[2].y : (j == 2 ? fl[2].z : fl[2].w));
            lb_collide_site<Real, Store, Shifted, Macro>(c, s0 + j, f[j], fo[j], fx, fy, fz, inv_in, scale_out, psum,
                                                        pmax, pbad, amax);
        }
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const Real v[4] = {fo[0][i], fo[1][i], fo[2][i], fo[3][i]};
            store4(c.fdst + (size_t)i * N + s0, v, 1.f);
        }
    }
    if (timed_out && threadIdx.x == 0) {
        atomicOr(&c.ctrl[2], 1u);
        // rows k .. k + kRowStages - 1 (those that exist) were issued and not consumed
        for (int q = k; q < k + kRowStages && q < my_rows; ++q)
            row_bar_wait(smem_addr(&full[q % kRowStages]), (uint32_t)(q / kRowStages) & 1u);
    }
    amax /= scale_out;  // back to population units for the controller
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    scale_controller_block(c, amax, scale_out, (int)gridDim.x, wmax, last);
}

size_t lb_rows_smem(int nx, int store_bytes)
{
    return (size_t)kRowStages * ((size_t)19 * nx * store_bytes + (size_t)3 * nx * sizeof(float));
}

bool lb_rows_valid(int nx, int store_bytes)
{
    return store_bytes == 2 && nx % (32 * kRowSPT) == 0 && nx <= kRowMaxNx;
}

// Resident blocks of one instantiation for rows of nx sites (the persistent
// grid), computed once per row length by lb_rows_prepare, outside any graph
// capture.
template <typename Real, typename Store, bool Shifted, int Macro>
int& rows_resident(int nx)
{
    static int resident[kRowMaxNx / (32 * kRowSPT) + 1] = {};
    return resident[nx / (32 * kRowSPT)];
}

template <typename Real, typename Store, bool Shifted, int Macro>
cudaError_t prepare_rows_one(int nx)
{
    int& resident = rows_resident<Real, Store, Shifted, Macro>(nx);
    if (resident > 0) return cudaSuccess;
    auto kern = lb_rows_kernel<Real, Store, Shifted, Macro>;
    const size_t smem = lb_rows_smem(nx, (int)sizeof(Store));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)lb_rows_smem(kRowMaxNx, 2));
    int dev = 0, sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nx / kRowSPT, smem);
    if (e == cudaSuccess) resident = (per_sm > 0 ? per_sm : 1) * sms;
    return e;
}

template <typename Store>
cudaError_t prepare_rows_store(int nx)
{
    cudaError_t e = prepare_rows_one<float, Store, true, 0>(nx);
    if (e == cudaSuccess) e = prepare_rows_one<float, Store, true, 1>(nx);
    if (e == cudaSuccess) e = prepare_rows_one<float, Store, false, 0>(nx);
    if (e == cudaSuccess) e = prepare_rows_one<float, Store, false, 1>(nx);
    return e;
}

cudaError_t lb_rows_prepare(int nx, int storage)
{
    if (!lb_rows_valid(nx, 2)) return cudaSuccess;
    if (storage == NH_STORE_F16S) return prepare_rows_store<__half>(nx);
    if (storage == NH_STORE_BF16S) return prepare_rows_store<__nv_bfloat16>(nx);
    return cudaSuccess;
}

template <typename Real, typename Store, bool Shifted, int Macro>
cudaError_t launch_lb_rows(const LBChan<Real, Store>& c, cudaStream_t st)
{
    const int resident = rows_resident<Real, Store, Shifted, Macro>(c.g.nx);
    if (resident <= 0) return cudaErrorNotReady;  // lb_rows_prepare was not run for this row length
    const int rows = c.g.ny * c.g.nz;
    const int blocks = rows < resident ? rows : resident;
    lb_rows_kernel<Real, Store, Shifted, Macro>
        <<<blocks, c.g.nx / kRowSPT, lb_rows_smem(c.g.nx, (int)sizeof(Store)), st>>>(c);
    return cudaGetLastError();
}

// Batched sweep: a persistent grid walks the (channel, tile) work list of up to
// kMaxBatch channels; tiles of channel k are [prefix[k], prefix[k+1]).
template <typename Real, typename Store, bool Shifted, bool WriteMacro, int SPT, bool Solid = false>
__global__ void __launch_bounds__(kLBThreads) lb_batch_kernel(const LBBatch<Real, Store> b)
{
    const int total = b.prefix[b.count];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        int lo = 0, hi = b.count - 1;  // channel k with prefix[k] <= t < prefix[k+1]
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (b.prefix[mid] <= t)
                lo = mid;
            else
                hi = mid - 1;
        }
        lb_tile<Real, Store, Shifted, WriteMacro ? 1 : 0, SPT, Solid>(b.ch[lo], t - b.prefix[lo],
                                                                     b.prefix[lo + 1] - b.prefix[lo]);
    }
}

// Launch variants: sites per thread x threads per block.
struct LBVariantShape {
    int spt, threads;
};
// The last variant, kLBRowsVariant, is lb_rows_kernel (16-bit stores only);
// its entry here is the two-site shape it falls back to where it does not apply.
constexpr LBVariantShape kLBVariants[kLBVariantCount] = {{2, 256}, {1, 256}, {2, 128}, {1, 128},
                                                         {4, 128}, {4, 64},  {2, 256}};

bool lb_variant_valid(int variant, int nx)
{
    if (variant < 0 || variant >= kLBVariantCount || variant == kLBRowsVariant) return false;
    return nx % kLBVariants[variant].spt == 0;
}

bool lb_variant_valid_for(int variant, int nx, int store_bytes)
{
    if (variant == kLBRowsVariant) return lb_rows_valid(nx, store_bytes);
    return lb_variant_valid(variant, nx);
}

int lb_blocks(int variant, int N)
{
    const LBVariantShape v = kLBVariants[variant];
    const int threads_needed = (N + v.spt - 1) / v.spt;
    return (threads_needed + v.threads - 1) / v.threads;
}

template <typename Real, typename Store, bool Shifted, int Macro>
cudaError_t launch_lb_spt(const LBChan<Real, Store>& c, int variant, cudaStream_t st)
{
    if constexpr (sizeof(Store) == 2 && Macro < 2) {
        if (variant == kLBRowsVariant && c.solid == nullptr && lb_rows_valid(c.g.nx, 2))
            return launch_lb_rows<Real, Store, Shifted, Macro>(c, st);
    }
    if (c.solid != nullptr) {  // obstacles: one site per thread, 256 threads
        if constexpr (Macro < 2)
            lb_kernel<Real, Store, Shifted, Macro, 1, true><<<(c.g.N + 255) / 256, 256, 0, st>>>(c);
        else
            return cudaErrorInvalidValue;
        return cudaGetLastError();
    }
    const LBVariantShape v = kLBVariants[variant];
    const int blocks = lb_blocks(variant, c.g.N);
    if (v.spt == 4)
        lb_kernel<Real, Store, Shifted, Macro, 4><<<blocks, v.threads, 0, st>>>(c);
    else if (v.spt == 2)
        lb_kernel<Real, Store, Shifted, Macro, 2><<<blocks, v.threads, 0, st>>>(c);
    else
        lb_kernel<Real, Store, Shifted, Macro, 1><<<blocks, v.threads, 0, st>>>(c);
    return cudaGetLastError();
}

template <typename Real, typename Store>
cudaError_t launch_lb(const LBChan<Real, Store>& c, bool shifted, bool write_macro, int variant, cudaStream_t st)
{
    if (!lb_variant_valid_for(variant, c.g.nx, (int)sizeof(Store))) return cudaErrorInvalidValue;
    if constexpr (sizeof(Store) != 2) {
        if (write_macro && c.part != nullptr) {
            if (c.solid != nullptr) return cudaErrorInvalidValue;
            return shifted ? launch_lb_spt<Real, Store, true, 2>(c, variant, st)
                           : launch_lb_spt<Real, Store, false, 2>(c, variant, st);
        }
    }
    if (shifted) {
        if (write_macro) return launch_lb_spt<Real, Store, true, 1>(c, variant, st);
        return launch_lb_spt<Real, Store, true, 0>(c, variant, st);
    }
    if (write_macro) return launch_lb_spt<Real, Store, false, 1>(c, variant, st);
    return launch_lb_spt<Real, Store, false, 0>(c, variant, st);
}

template <typename Real, typename Store, bool Shifted, bool WriteMacro>
cudaError_t launch_lb_batch_spt(LBBatch<Real, Store>& b, int variant, int grid, cudaStream_t st)
{
    bool solid = false;
    for (int k = 0; k < b.count; ++k) solid = solid || b.ch[k].solid != nullptr;
    if (solid) {  // obstacles in the batch: one site per thread, 256 threads, for every channel
        b.prefix[0] = 0;
        for (int k = 0; k < b.count; ++k) b.prefix[k + 1] = b.prefix[k] + (b.ch[k].g.N + 255) / 256;
        const int blocks = grid < b.prefix[b.count] ? grid : b.prefix[b.count];
        lb_batch_kernel<Real, Store, Shifted, WriteMacro, 1, true><<<blocks, 256, 0, st>>>(b);
        return cudaGetLastError();
    }
    const LBVariantShape v = kLBVariants[variant];
    b.prefix[0] = 0;
    for (int k = 0; k < b.count; ++k) {
        const int threads_needed = (b.ch[k].g.N + v.spt - 1) / v.spt;
        b.prefix[k + 1] = b.prefix[k] + (threads_needed + v.threads - 1) / v.threads;
    }
    const int blocks = grid < b.prefix[b.count] ? grid : b.prefix[b.count];
    if (v.spt == 4)
        lb_batch_kernel<Real, Store, Shifted, WriteMacro, 4><<<blocks, v.threads, 0, st>>>(b);
    else if (v.spt == 2)
        lb_batch_kernel<Real, Store, Shifted, WriteMacro, 2><<<blocks, v.threads, 0, st>>>(b);
    else
        lb_batch_kernel<Real, Store, Shifted, WriteMacro, 1><<<blocks, v.threads, 0, st>>>(b);
    return cudaGetLastError();
}

template <typename Real, typename Store>
cudaError_t launch_lb_batch(LBBatch<Real, Store>& b, bool shifted, bool write_macro, int variant, int grid,
                            cudaStream_t st)
{
    if (b.count < 1 || b.count > kMaxBatch) return cudaErrorInvalidValue;
    for (int k = 0; k < b.count; ++k)
        if (!lb_variant_valid(variant, b.ch[k].g.nx)) return cudaErrorInvalidValue;
    if (shifted) {
        if (write_macro) return launch_lb_batch_spt<Real, Store, true, true>(b, variant, grid, st);
        return launch_lb_batch_spt<Real, Store, true, false>(b, variant, grid, st);
    }
    if (write_macro) return launch_lb_batch_spt<Real, Store, false, true>(b, variant, grid, st);
    return launch_lb_batch_spt<Real, Store, false, false>(b, variant, grid, st);
}

template cudaError_t launch_lb_batch<double, double>(LBBatch<double, double>&, bool, bool, int, int, cudaStream_t);
template cudaError_t launch_lb_batch<float, float>(LBBatch<float, float>&, bool, bool, int, int, cudaStream_t);
template cudaError_t launch_lb_batch<float, __half>(LBBatch<float, __half>&, bool, bool, int, int, cudaStream_t);
template cudaError_t launch_lb_batch<float, __nv_bfloat16>(LBBatch<float, __nv_bfloat16>&, bool, bool, int, int,
                                                           cudaStream_t);

template cudaError_t launch_lb<double, double>(const LBChan<double, double>&, bool, bool, int, cudaStream_t);
template cudaError_t launch_lb<float, float>(const LBChan<float, float>&, bool, bool, int, cudaStream_t);
template cudaError_t launch_lb<float, __half>(const LBChan<float, __half>&, bool, bool, int, cudaStream_t);
template cudaError_t launch_lb<float, __nv_bfloat16>(const LBChan<float, __nv_bfloat16>&, bool, bool, int,
                                                     cudaStream_t);

}  // namespace nh
