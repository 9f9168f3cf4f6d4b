// nh_internal.cuh -- device-side building blocks and launch interfaces of the
// hybrid LB + FD nematohydrodynamics library (arXiv:2503.06610).  Shared by
// the kernel translation units and the C-ABI layer; not part of the public ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/nh.h"

namespace nh {

// ------------------------------------------------------------------ D3Q19
// Velocity order of the public header (rest, +-x, +-y, +-z, xy, xz, yz pairs).
// Weights 1/3, 1/18, 1/36 and c_s^2 = 1/3 (Sec. II.C).
#define NH_D3Q19_TABLES                                                                                 \
    constexpr int EX[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};           \
    constexpr int EY[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};           \
    constexpr int EZ[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};           \
    constexpr int OPP[19] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};      \
    (void)EX; (void)EY; (void)EZ; (void)OPP;

template <typename Real>
__device__ __forceinline__ Real d3q19_w(int i)
{
    return i == 0 ? Real(1) / Real(3) : (i < 7 ? Real(1) / Real(18) : Real(1) / Real(36));
}

// ------------------------------------------------------------------ storage codecs
// Populations are stored as Store and computed as Real.  The 16-bit codecs hold
// 2^k * f_shifted; `scale` = 2^k and `inv_scale` = 2^-k (exact powers of two).
template <typename Store, typename Real>
struct Codec;

template <>
struct Codec<double, double> {
    static __device__ __forceinline__ double load(const double* p, float) { return *p; }
    static __device__ __forceinline__ void store(double* p, double v, float) { *p = v; }
};
template <>
struct Codec<float, float> {
    static __device__ __forceinline__ float load(const float* p, float) { return *p; }
    static __device__ __forceinline__ void store(float* p, float v, float) { *p = v; }
};
template <>
struct Codec<__half, float> {
    static __device__ __forceinline__ float load(const __half* p, float inv_scale)
    {
        return __half2float(*p) * inv_scale;
    }
    static __device__ __forceinline__ void store(__half* p, float v, float scale) { *p = __float2half_rn(v * scale); }
};
template <>
struct Codec<__nv_bfloat16, float> {
    static __device__ __forceinline__ float load(const __nv_bfloat16* p, float inv_scale)
    {
        return __bfloat162float(*p) * inv_scale;
    }
    static __device__ __forceinline__ void store(__nv_bfloat16* p, float v, float scale)
    {
        *p = __float2bfloat16_rn(v * scale);
    }
};

// ------------------------------------------------------------------ geometry
struct Geom {
    int nx, ny, nz;
    int walls;      // bounce-back plates in z
    int anchoring;  // NH_ANCHOR_*
    int N;          // nx*ny*nz
};

__device__ __forceinline__ int wrap_p(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// ------------------------------------------------------------------ LB
// One channel's LB sweep arguments.  For the 16-bit stores `scales` points to
// four device floats: [0], [1] = scale 2^k of the data in population buffer
// 0 / 1, [2] = target scale for the next write; `ctrl` to two words used by
// the in-kernel scale controller (running max |f*| as float bits, and a
// block-completion ticket).
template <typename Real, typename Store>
struct LBChan {
    const Store* fsrc;
    Store* fdst;
    const Real* F;  // [3][N] F_lc, frozen over the FD interval
    const Real* Fu; // [3][N] F_lc whose half shifts u, or null: F (paper ordering of Sec. II.D)
    const unsigned char* solid;  // [N] 1 = solid node (obstacle), or null: none
    Real* u;        // [3][N] written on macro steps
    Real* rho;      // [N]    written on macro steps
    float* scales;
    unsigned* ctrl;
    double* part;   // [3][blocks] diagnostics partials of a macro launch, or null (F32 / F64 stores)
    int src;        // index (0/1) of the source buffer
    Geom g;
    Real omega;     // 1/tau
    Real gx, gy, gz;
};

// Scaled 16-bit stores keep max |2^k f*| near 2^kScaleHeadroomLog2.
constexpr int kScaleHeadroomLog2 = 12;

// ------------------------------------------------------------------ FD
template <typename Real>
struct FDPar {
    Real K, q0, W0;
    Real inv_gamma1, gamma2, g2_over_g1;
    Real a1, a2, a3, a4p, a5, a6;
    Real dt;
    Real kd1, kd2, kd3;  // K11 - K, K22 - K, K33 - K (three-constant energy)
    // The same constants with the factors 1/2 of the central differences and
    // of the strain-rate and vorticity tensors folded in (lambda = g2/g1):
    Real kg, kqg, w0g, c1, c2;            // K/g1, K q0/g1, W0/g1, (1 - lambda)/4, -(1 + lambda)/4
    Real kq, g2q, a1q, a4q, a5q, a6q, k4, kq2;  // K q0, lambda/4, a1/4, a4'/4, a5/4, a6/4, K/4, K q0/2
    // Reading flags (nh_params): renormalise the predictor; central-of-central
    // second derivatives in h (per-site kernels); N of the stress from the
    // corrector's averaged rate, which the corrector then leaves in ndot
    // (per-site kernels; set only for the force that follows an FD update);
    // ghost stress = the adjacent layer's in the force divergence.
    int renorm_p, lap_wide, n_rate, mirror;
};

// Three-constant correction of the Frank energy density at one site
// (Eq. free-energy-eq minus its one-constant form with K), from the director
// n and its central gradient G[b][c] = d_b n_c:
//   div = G_aa, w = curl n (w_a = eps_abc G_bc), t = n.w + q0,
//   df = kd1/2 div^2 + kd2/2 t^2 + kd3/2 (|n|^2 |w|^2 - (n.w)^2).
// Writes dfdn[c] = d df/d n_c and P[b][c] = d df/d G_bc; returns df.
template <typename Real>
__device__ __forceinline__ Real frank3_site(const Real n[3], const Real G[3][3], Real kd1, Real kd2, Real kd3,
                                                    Real q0, Real dfdn[3], Real P[3][3])
{
    const Real div = G[0][0] + G[1][1] + G[2][2];
    const Real w[3] = {G[1][2] - G[2][1], G[2][0] - G[0][2], G[0][1] - G[1][0]};
    const Real nw = n[0] * w[0] + n[1] * w[1] + n[2] * w[2];
    const Real nn = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
    const Real ww = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    const Real t = nw + q0;
    Real V[3];  // d df / d w
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        dfdn[c] = kd2 * t * w[c] + kd3 * (n[c] * ww - nw * w[c]);
        V[c] = kd2 * t * n[c] + kd3 * (nn * w[c] - nw * n[c]);
    }
    // P[b][c] = kd1 div delta_bc + eps_abc V_a
    P[0][0] = kd1 * div;
    P[1][1] = kd1 * div;
    P[2][2] = kd1 * div;
    P[1][2] = V[0];
    P[2][1] = -V[0];
    P[2][0] = V[1];
    P[0][2] = -V[1];
    P[0][1] = V[2];
    P[1][0] = -V[2];
    return Real(0.5) * kd1 * div * div + Real(0.5) * kd2 * t * t + Real(0.5) * kd3 * (nn * ww - nw * nw);
}

template <typename Real>
struct FDChan {
    Real* n;      // [3][N] director (in place on the corrector)
    Real* nP;     // [3][N] predictor
    Real* ndot;   // [3][N] (dn/dt)_old
    const Real* u;   // [3][N]
    Real* sigma;  // [9][N]
    Real* F;      // [3][N] F_lc
    Real* P3;     // [9][N] d df/d(d_b n_c) of the three-constant correction, or null (one constant)
    const unsigned char* solid;  // [N] 1 = solid node (obstacle), or null: none
    Geom g;
    FDPar<Real> p;
    int zch = 0;  // layers per chunk of the fused kernels; 0: chosen from g alone
};

// Diagnostics folded into the stress kernel (fused B) of an FD update that
// follows a macro LB launch: per-block partials of the lattice Frank energy,
// the |n| extrema, the non-finite director count and the tube sums of the
// updated director, laid out as the diagnostics kernels' partials
// ([V][blocks]), each block also taking its slice of the LB launch's
// population, max |u| and non-finite partials.
struct BDiag {
    const double* tubes;   // [n_tubes][2] previous centroids (device)
    int n_tubes;
    const double* trig;    // FP64 sin/cos tables of the column positions
    double* partials;
    const double* lbpart;  // [3][lbp_blocks]
    int lbp_blocks;
};

// ------------------------------------------------------------------ launchers (host)
// Batched launches: up to kMaxBatch channel descriptors travel as kernel
// parameters (no device allocation); prefix[k] is the first tile of channel k.
constexpr int kMaxBatch = 64;
template <typename Real, typename Store>
struct LBBatch {
    int count;
    int prefix[kMaxBatch + 1];
    LBChan<Real, Store> ch[kMaxBatch];
};
template <typename Real>
struct FDBatch {
    int count;
    int prefix[kMaxBatch + 1];
    FDChan<Real> ch[kMaxBatch];
};

// LB launch variants (sites per thread x block size); variant 0 is the default.
constexpr int kLBVariantCount = 7;
constexpr int kLBRowsVariant = 6;  // rows staged in shared memory by bulk copies (16-bit stores)
bool lb_variant_valid(int variant, int nx);  // the register shapes 0 .. 5 (also in batches)
bool lb_rows_valid(int nx, int store_bytes);
bool lb_variant_valid_for(int variant, int nx, int store_bytes);  // any variant, one channel
cudaError_t lb_rows_prepare(int nx, int storage);  // once per context, outside graph capture
int lb_blocks(int variant, int N);  // thread blocks of one LB launch of that shape
template <typename Real, typename Store>
cudaError_t launch_lb(const LBChan<Real, Store>& c, bool shifted, bool write_macro, int variant, cudaStream_t s);

// Batched LB sweep over b.count channels with a persistent grid of at most
// `grid` blocks (fills b.prefix).
template <typename Real, typename Store>
cudaError_t launch_lb_batch(LBBatch<Real, Store>& b, bool shifted, bool write_macro, int variant, int grid,
                            cudaStream_t s);

// Batched FD kernels: stage 0 predict, 1 correct, 2 stress, 3 force.
template <typename Real>
cudaError_t launch_fd_batch(FDBatch<Real>& b, int stage, int grid, cudaStream_t s);

// Fused FD kernels (2.5D shared-memory tiles): A = predictor + corrector +
// renormalisation (nin, u -> nout), B = stress + force (nin, u -> F; copies
// nin into ncopy when ncopy is not null); batched stages 0 = A (n -> nP),
// 1 = B (nP -> F, n), 2 = A (nP -> n).
template <typename Real>
cudaError_t launch_fd_fused_a(const FDChan<Real>& c, const Real* nin, Real* nout, cudaStream_t s);
template <typename Real>
cudaError_t launch_fd_fused_b(const FDChan<Real>& c, const Real* nin, Real* ncopy, cudaStream_t s,
                              const BDiag* diag = nullptr);
template <typename Real>
int fd_fused_tiles(const FDChan<Real>& c);  // blocks of a single-channel fused launch
template <typename Real>
cudaError_t launch_fd_fused_batch(FDBatch<Real>& b, int stage, int grid, cudaStream_t s);

template <typename Real>
cudaError_t launch_fd_predict(const FDChan<Real>& c, cudaStream_t s);
template <typename Real>
cudaError_t launch_fd_correct(const FDChan<Real>& c, cudaStream_t s);
template <typename Real>
cudaError_t launch_stress(const FDChan<Real>& c, cudaStream_t s);
template <typename Real>
cudaError_t launch_force(const FDChan<Real>& c, cudaStream_t s);
// P = d df/d(d_b n_c) of the three-constant correction from n (or n^P) into c.P3
template <typename Real>
cudaError_t launch_frank3_p(const FDChan<Real>& c, bool from_predictor, cudaStream_t s);

// Field conversion and initialisation (diag.cu)
template <typename Real>
cudaError_t launch_load_fields(const double* n, const double* u, const double* rho, Real* dn, Real* du, Real* drho,
                               int N, cudaStream_t s);
template <typename Real>
cudaError_t launch_store_vec(const Real* src, double* dst, int64_t count, cudaStream_t s);
template <typename Real, typename Store>
cudaError_t launch_init_populations(const Real* rho, const Real* u, Store* f, const float* scale, int N, bool shifted,
                                    cudaStream_t s);
template <typename Store>
cudaError_t launch_decode_plane(const Store* f, double* dst, int N, const float* scale, cudaStream_t s);
template <typename Store>
cudaError_t launch_encode_plane(const double* src, Store* f, int N, const float* scale, cudaStream_t s);

cudaError_t launch_scale_init(const float* rho, const float* u, const float* F, const double g[3], int N,
                              float* scales, unsigned* ctrl, cudaStream_t s);

// Diagnostics (diag.cu)
struct DiagArgs {
    const void* f;      // populations (Store)
    int storage;
    int shifted;
    const void* n;      // Real [3][N]
    const void* u;
    const void* rho;
    int precision;
    const float* scale;
    Geom g;
    double K, q0, W0;
    int frank3;         // add the three-constant correction to the energy
    const unsigned char* solid;  // [N] 1 = solid node: excluded from the sums (links to fluid kept), or null
    double kd1, kd2, kd3;
    int n_tubes;
    double tubes[NH_MAX_TUBES][2];
    const double* trig; // [sin x | cos x | sin y | cos y] of 2 pi x/nx, 2 pi y/ny
    double* partials;   // [blocks][NDIAG]
    double* result;     // [NDIAG]
    int blocks;
    // [3][lbp_blocks] mass, max |u| and non-finite partials left by the LB launch that
    // wrote f, u and rho (F32 / F64 stores, no obstacles): only n is read; or null
    const double* lbpart = nullptr;
    int lbp_blocks = 0;
};
int diag_num_values(int n_tubes);
int diag_blocks();
cudaError_t launch_diagnostics(const DiagArgs& a, cudaStream_t s);
// The final reduction alone, over partials [V][blocks] that another kernel left.
cudaError_t launch_diag_final(const double* partials, double* result, int blocks, int V, cudaStream_t s);
cudaError_t launch_trig_table(double* t, int nx, int ny, cudaStream_t s);

// max |n - snap| over sites into *out (device), then snap <- n (diag.cu)
template <typename Real>
cudaError_t launch_director_change(const Real* n, Real* snap, double* partial, double* out, int N, cudaStream_t s);

// C4 projection of the director about the axis through (nx/2, nx/2) (diag.cu)
template <typename Real>
cudaError_t launch_symmetrize_c4(const Real* n, Real* out, int nx, int nz, cudaStream_t s);

// Row copies between slabs (slab.cu): item k copies `comps` components of
// one row (nz runs of nx consecutive elements) from src to dst; component c,
// layer z starts at c * cstride + z * zstride elements from the base.
constexpr int kMaxRowCopies = 96;
constexpr int kMaxSlabs = 64;
struct RowCopyItem {
    const void* src;
    void* dst;
    int nx, nz, comps;
    int src_zstride, dst_zstride;
    int src_cstride, dst_cstride;
};
struct RowCopyList {
    int count;
    RowCopyItem item[kMaxRowCopies];
};
cudaError_t launch_row_copies(const RowCopyList& list, int elem_bytes, cudaStream_t s);

// The parameter checks of nh_create (api.cu): NH_OK, or NH_EINVAL with the reason in err.
int validate_params(const nh_params* p, std::string& err);

// Record the text returned by nh_last_error(NULL) on this thread (api.cu).
void set_global_error(const char* msg);
inline void set_global_error(const std::string& msg) { set_global_error(msg.c_str()); }

}  // namespace nh
