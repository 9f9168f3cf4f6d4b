// lb.cu -- fused D3Q19 lattice-Boltzmann collide-and-stream sweep
// (arXiv:2503.06610, Sec. II.C).
//
// One thread owns one site and performs, in registers:
//   1. streaming by pull: f_i(x) <- f*_i(x - e_i) of the previous step, or the
//      half-way bounce-back f*_opp(i)(x) when x - e_i lies in a plate;
//   2. moments, Eqs. shifted-rho / shifeted-u (or the plain ones):
//      rho - 1 = sum_i f^s_i,  rho u = sum_i e_i f^s_i + F/2,  F = F_lc + rho g;
//   3. equilibrium (Eq. shifted-feq or Eq. feq-eq) and Guo source S_i^F;
//   4. SRT relaxation (Eq. shifted-lbe): f*_i = f_i - (f_i - f^eq_i)/tau
//      + (1 - 1/(2 tau)) S_i^F, written to the other population buffer.
// Populations are structure-of-arrays planes [19][N] so every warp reads and
// writes 19 runs of consecutive sites (x fastest): coalesced, with the +-1 x
// shift of the pulled planes served from L1/L2.  u and rho are written only on
// steps that feed an FD update (or end a call).
#include "nh_internal.cuh"

namespace nh {

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

template <typename Real, typename Store, bool Shifted, bool WriteMacro>
__global__ void __launch_bounds__(256) lb_kernel(const LBChan<Real, Store> c)
{
    NH_D3Q19_TABLES
    constexpr bool kScaled = sizeof(Store) == 2;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = c.g.N;
    float amax = 0.f;
    float scale_out = 1.f;
    if (kScaled) scale_out = c.scales[2];
    if (s < N) {
        const int nx = c.g.nx, ny = c.g.ny, nz = c.g.nz;
        const int x = s % nx;
        const int t = s / nx;
        const int y = t % ny;
        const int z = t / ny;
        const float inv_in = kScaled ? 1.f / c.scales[c.src] : 1.f;

        // 1. pull streaming with half-way bounce-back
        Real f[19];
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const int zs = z - EZ[i];
            size_t off;
            if (EZ[i] != 0 && c.g.walls && (zs < 0 || zs >= nz)) {
                off = (size_t)OPP[i] * N + s;
            } else {
                const int xs = wrap_p(x - EX[i], nx);
                const int ys = wrap_p(y - EY[i], ny);
                const int zz = wrap_p(zs, nz);
                off = (size_t)i * N + (xs + nx * (ys + ny * zz));
            }
            f[i] = Codec<Store, Real>::load(c.fsrc + off, inv_in);
        }

        // 2. moments
        Real sum = 0, mx = 0, my = 0, mz = 0;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            sum += f[i];
            if (EX[i] != 0) mx += EX[i] > 0 ? f[i] : -f[i];
            if (EY[i] != 0) my += EY[i] > 0 ? f[i] : -f[i];
            if (EZ[i] != 0) mz += EZ[i] > 0 ? f[i] : -f[i];
        }
        const Real rho = Shifted ? Real(1) + sum : sum;
        const Real drho = Shifted ? sum : sum - Real(1);
        const Real Fx = c.F[s] + rho * c.gx;
        const Real Fy = c.F[N + s] + rho * c.gy;
        const Real Fz = c.F[2 * N + s] + rho * c.gz;
        const Real inv_rho = Real(1) / rho;
        const Real ux = (mx + Real(0.5) * Fx) * inv_rho;
        const Real uy = (my + Real(0.5) * Fy) * inv_rho;
        const Real uz = (mz + Real(0.5) * Fz) * inv_rho;
        if (WriteMacro) {
            c.u[s] = ux;
            c.u[N + s] = uy;
            c.u[2 * N + s] = uz;
            c.rho[s] = rho;
        }

        // 3-4. equilibrium, Guo source, relaxation
        const Real omega = c.omega;
        const Real cS = Real(1) - Real(0.5) * omega;
        const Real uu = ux * ux + uy * uy + uz * uz;
        const Real uF = ux * Fx + uy * Fy + uz * Fz;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const Real w = d3q19_w<Real>(i);
            const Real eu = Real(EX[i]) * ux + Real(EY[i]) * uy + Real(EZ[i]) * uz;
            const Real eF = Real(EX[i]) * Fx + Real(EY[i]) * Fy + Real(EZ[i]) * Fz;
            Real feq = w * rho * (Real(3) * eu + Real(4.5) * eu * eu - Real(1.5) * uu);
            feq += Shifted ? w * drho : w * rho;
            const Real S = w * (Real(3) * eF + Real(9) * eu * eF - Real(3) * uF);
            const Real fo = f[i] + omega * (feq - f[i]) + cS * S;
            if (kScaled) amax = fmaxf(amax, fabsf((float)fo));
            Codec<Store, Real>::store(c.fdst + (size_t)i * N + s, fo, scale_out);
        }
    }
    if (kScaled) {
        // In-kernel scale controller: block max -> global running max; the last
        // block to finish records the scale of the buffer just written and sets
        // the target of the next step from this step's max |f*|.
        __shared__ float wmax[8];
        __shared__ bool last;
        for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = amax;
        __syncthreads();
        if (threadIdx.x == 0) {
            float b = 0.f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = fmaxf(b, wmax[w]);
            if (b > __int_as_float((int)__ldcg(&c.ctrl[0]))) atomicMax(reinterpret_cast<int*>(&c.ctrl[0]), __float_as_int(b));
            __threadfence();
            const unsigned ticket = atomicAdd(&c.ctrl[1], 1u);
            last = ticket == gridDim.x - 1;
        }
        __syncthreads();
        if (last && threadIdx.x == 0) {
            __threadfence();
            const float m = __int_as_float((int)atomicExch(&c.ctrl[0], 0u));
            c.scales[1 - c.src] = scale_out;
            c.scales[2] = scale_for(m, scale_out);
            c.ctrl[1] = 0u;
        }
    }
}

template <typename Real, typename Store>
cudaError_t launch_lb(const LBChan<Real, Store>& c, bool shifted, bool write_macro, cudaStream_t st)
{
    const int threads = 256;
    const int blocks = (c.g.N + threads - 1) / threads;
    if (shifted) {
        if (write_macro)
            lb_kernel<Real, Store, true, true><<<blocks, threads, 0, st>>>(c);
        else
            lb_kernel<Real, Store, true, false><<<blocks, threads, 0, st>>>(c);
    } else {
        if (write_macro)
            lb_kernel<Real, Store, false, true><<<blocks, threads, 0, st>>>(c);
        else
            lb_kernel<Real, Store, false, false><<<blocks, threads, 0, st>>>(c);
    }
    return cudaGetLastError();
}

template cudaError_t launch_lb<double, double>(const LBChan<double, double>&, bool, bool, cudaStream_t);
template cudaError_t launch_lb<float, float>(const LBChan<float, float>&, bool, bool, cudaStream_t);
template cudaError_t launch_lb<float, __half>(const LBChan<float, __half>&, bool, bool, cudaStream_t);
template cudaError_t launch_lb<float, __nv_bfloat16>(const LBChan<float, __nv_bfloat16>&, bool, bool, cudaStream_t);

}  // namespace nh
