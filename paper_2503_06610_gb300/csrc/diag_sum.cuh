// diag_sum.cuh -- device pieces of the global diagnostics reduction shared by
// the diagnostics kernels and the stress kernel that folds them in: warp
// reductions, the lattice link energy, the tube assignment and sums, and the
// per-block partials (FP64 across warps in a fixed order).
#pragma once

#include "nh_internal.cuh"

namespace nh {
namespace dsum {

constexpr int DIAG_THREADS = 256;
constexpr int DIAG_FIXED = 6;  // mass, energy, max_u, min_norm, max_norm, nonfinite

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_min(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// |v| of a 3-vector, one expression for every kernel that reports extrema of
// it; the fused multiply-adds are explicit, so no kernel's inlining context
// can contract it differently.
template <typename Real>
__device__ __forceinline__ Real norm3(const Real v[3])
{
    return sqrt(fma(v[2], v[2], fma(v[1], v[1], v[0] * v[0])));
}

// Energy of the link from n (at x) to m (at x + e_b):
// K/2 |m - n|^2 + K q0 eps_abc n_a m_c  (= K/2 |m - n|^2 - K q0 (n x m)_b).
template <typename Real>
__device__ __forceinline__ Real link_energy(const Real n[3], const Real m[3], int b, Real K, Real q0)
{
    const Real d0 = m[0] - n[0], d1 = m[1] - n[1], d2 = m[2] - n[2];
    Real cr;
    if (b == 0)
        cr = n[1] * m[2] - n[2] * m[1];
    else if (b == 1)
        cr = n[2] * m[0] - n[0] * m[2];
    else
        cr = n[0] * m[1] - n[1] * m[0];
    return Real(0.5) * K * (d0 * d0 + d1 * d1 + d2 * d2) - K * q0 * cr;
}

// Nearest previous tube centroid of column (x, y) (-1 without tubes): FP32
// squared distances with the periodic minimum image; a near-tie of the two
// best is settled in FP64 so that the choice equals the FP64 one.
__device__ __forceinline__ int nearest_tube(const Geom& g, const double* tubes, const float (*txy)[2], int T, int x,
                                            int y)
{
    int owner = -1, second = -1;
    float bd = 3.0e38f, bd2 = 3.0e38f;
    const float hx = 0.5f * g.nx, hy = 0.5f * g.ny;
    for (int k = 0; k < T; ++k) {
        float dx = (float)x - txy[k][0], dy = (float)y - txy[k][1];
        dx = dx > hx ? dx - g.nx : (dx < -hx ? dx + g.nx : dx);
        dy = dy > hy ? dy - g.ny : (dy < -hy ? dy + g.ny : dy);
        const float d2 = dx * dx + dy * dy;
        if (d2 < bd) {
            bd2 = bd;
            second = owner;
            bd = d2;
            owner = k;
        } else if (d2 < bd2) {
            bd2 = d2;
            second = k;
        }
    }
    if (second >= 0 && bd2 - bd <= 1e-3f * (1.f + bd)) {
        double d2[2];
        const int cand[2] = {owner, second};
        for (int j = 0; j < 2; ++j) {
            double dx = x - tubes[2 * cand[j]], dy = y - tubes[2 * cand[j] + 1];
            dx = dx > 0.5 * g.nx ? dx - g.nx : (dx < -0.5 * g.nx ? dx + g.nx : dx);
            dy = dy > 0.5 * g.ny ? dy - g.ny : (dy < -0.5 * g.ny ? dy + g.ny : dy);
            d2[j] = dx * dx + dy * dy;
        }
        // lowest index wins an exact tie, as in a first-minimum search
        if (d2[1] < d2[0] || (d2[1] == d2[0] && cand[1] < cand[0])) owner = cand[1];
    }
    return owner;
}

// Centroid sums of one column with tube weight wsum: wsum and wsum times
// sin / cos of 2 pi x / nx and 2 pi y / ny (FP64 tables in the FP64 build,
// sincospi in FP32 in the FP32 build).
template <typename Real>
__device__ __forceinline__ void tube_values(const Geom& g, const double* trig, int x, int y, Real wsum, Real v[5])
{
    v[0] = wsum;
    if (sizeof(Real) == 8) {
        v[1] = wsum * Real(trig[x]);                    // sin(2 pi x / nx)
        v[2] = wsum * Real(trig[g.nx + x]);             // cos(2 pi x / nx)
        v[3] = wsum * Real(trig[2 * g.nx + y]);         // sin(2 pi y / ny)
        v[4] = wsum * Real(trig[2 * g.nx + g.ny + y]);  // cos(2 pi y / ny)
    } else {
        float sx, cx, sy, cy;
        sincospif(2.f * (float)x / (float)g.nx, &sx, &cx);
        sincospif(2.f * (float)y / (float)g.ny, &sy, &cy);
        v[1] = wsum * Real(sx);
        v[2] = wsum * Real(cx);
        v[3] = wsum * Real(sy);
        v[4] = wsum * Real(cy);
    }
}

// Adds each lane's five tube values to its owner's row of the warp's
// accumulator (lane 0 writes; one warp sum per distinct owner in the warp).
// Every lane of the warp calls it (owner -1: nothing to add).
template <typename Real>
__device__ __forceinline__ void warp_tube_accumulate(int owner, const Real v[5], int lane, Real* acc)
{
    unsigned pending = __ballot_sync(0xffffffffu, owner >= 0);
    while (pending) {
        const int t = __shfl_sync(0xffffffffu, owner, __ffs(pending) - 1);
        const bool mine = owner == t;
        pending &= ~__ballot_sync(0xffffffffu, mine);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const Real sum = warp_sum(mine ? v[k] : Real(0));
            if (lane == 0) acc[t * 5 + k] += sum;
        }
    }
}

// Block partials, value-major (partials[k * gridDim.x + block]): FP64 sums
// of the threads' mass and energy, extrema, NaN count, then the tube sums
// combined across the block's warps in a fixed order.
template <int Threads = DIAG_THREADS, typename Real>
__device__ __forceinline__ void block_partials(double* partials, const double* lbpart, int lbp_blocks, Real mass_t,
                                               Real energy_t, Real max_u,
                                                    Real min_nn, Real max_nn, int bad,
                                                    const Real (*tube_acc)[NH_MAX_TUBES * 5], int T)
{
    __shared__ double red[Threads / 32][DIAG_FIXED];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // within a warp: sums in the build's precision, extrema exactly, the count
    // in integers (GB300's FP64 pipe is narrow); FP64 across the warps below
    const double mass = (double)warp_sum(mass_t);
    const double energy = (double)warp_sum(energy_t);
    const double dbad = (double)__reduce_add_sync(0xffffffffu, (unsigned)bad);
    Real mu = max_u, mn = min_nn, mx = max_nn;
    for (int o = 16; o > 0; o >>= 1) {
        mu = max(mu, __shfl_xor_sync(0xffffffffu, mu, o));
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const double dmax_u = (double)mu, dmin_nn = (double)mn, dmax_nn = (double)mx;
    if (lane == 0) {
        red[wid][0] = mass;
        red[wid][1] = energy;
        red[wid][2] = dmax_u;
        red[wid][3] = dmin_nn;
        red[wid][4] = dmax_nn;
        red[wid][5] = dbad;
    }
    // With lbpart, block b also takes its slice of the LB launch's block
    // partials (mass, max |u|, non-finite count): warp 0, lanes striding, then
    // a warp reduction, so the order is fixed.
    __shared__ double lbv[3];
    if (lbpart != nullptr && wid == 0) {
        const int nb = lbp_blocks;
        const int per = (nb + gridDim.x - 1) / gridDim.x;
        const int b0 = blockIdx.x * per, b1 = min(b0 + per, nb);
        double s0 = 0.0, m1 = 0.0, s2 = 0.0;
        for (int b = b0 + lane; b < b1; b += 32) {
            s0 += __ldg(lbpart + b);
            m1 = fmax(m1, __ldg(lbpart + nb + b));
            s2 += __ldg(lbpart + 2 * (size_t)nb + b);
        }
        s0 = warp_sum(s0);
        m1 = warp_max(m1);
        s2 = warp_sum(s2);
        if (lane == 0) {
            lbv[0] = s0;
            lbv[1] = m1;
            lbv[2] = s2;
        }
    }
    __syncthreads();
    double* out = partials + blockIdx.x;
    const size_t stride = gridDim.x;
    if (threadIdx.x == 0) {
        double v[DIAG_FIXED] = {0.0, 0.0, 0.0, 1e300, 0.0, 0.0};
        for (int w = 0; w < Threads / 32; ++w) {
            v[0] += red[w][0];
            v[1] += red[w][1];
            v[2] = fmax(v[2], red[w][2]);
            v[3] = fmin(v[3], red[w][3]);
            v[4] = fmax(v[4], red[w][4]);
            v[5] += red[w][5];
        }
        if (lbpart != nullptr) {
            v[0] += lbv[0];
            v[2] = fmax(v[2], lbv[1]);
            v[5] += lbv[2];
        }
        for (int k = 0; k < DIAG_FIXED; ++k) out[k * stride] = v[k];
    }
    for (int k = threadIdx.x; k < 5 * T; k += blockDim.x) {
        double acc = 0.0;
        for (int w = 0; w < Threads / 32; ++w) acc += (double)tube_acc[w][k];  // fixed order
        out[(DIAG_FIXED + k) * stride] = acc;
    }
}

}  // namespace dsum
}  // namespace nh
