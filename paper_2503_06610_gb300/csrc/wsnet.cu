// wsnet.cu -- the learned warm start: a 3D U-Net that maps the extruded
// skyrmion-tube ansatz (plus q0, Lz, W0) to the relaxed director field, with
// hand-written BF16 training and inference kernels (FP32 accumulation).
//
// Network (4 levels, widths 16/16/32/64, 394 419 parameters): two 3x3x3
// convolutions + ReLU per level, 2x2x2 mean pooling down, nearest x2 upsampling
// and channel concatenation up, a 1x1x1 head 16 -> 3 whose output corrects the
// ansatz, n = normalise(n_ansatz + delta).  Convolutions are cross-correlations,
// periodic in x and y and zero-padded in z.
//
// Layouts: activations are channels-last BF16 [batch][z][y][x][c]; activation
// gradients are channels-last FP32.  Parameters are one flat FP32 vector, layer
// by layer W[tap][cout][cin] (tap = 9 kz + 3 ky + kx) then bias[cout]; the head
// is W[3][16] then bias[3].
//
// Convolutions run on the tensor cores as implicit GEMMs (BF16 inputs, FP32
// accumulators):
//   forward       M = voxels (128 per CTA), N = cout, K = 27 taps x cin, on the
//                 5th-generation tensor cores (tcgen05.mma, accumulator in TMEM)
//   data grad     M = voxels, N = cin, K = 27 taps x cout (transposed weights),
//                 mma.sync.m16n8k16
//   weight grad   M = cout, N = cin, K = voxels (per tap; shared-memory tiles,
//                 FP32 atomics across voxel chunks), mma.sync.m16n8k16
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "nh_internal.cuh"

namespace {

using bf16 = __nv_bfloat16;

// ------------------------------------------------------------------ architecture

struct LayerDesc {
    int cin, cout;
};
constexpr int kLayers = 14;
constexpr LayerDesc kConv[kLayers] = {{16, 16}, {16, 16}, {16, 16}, {16, 16}, {16, 32}, {32, 32}, {32, 64},
                                      {64, 64}, {96, 32}, {32, 32}, {48, 16}, {16, 16}, {32, 16}, {16, 16}};
enum { ENC1A, ENC1B, ENC2A, ENC2B, ENC3A, ENC3B, BOTA, BOTB, DEC3A, DEC3B, DEC2A, DEC2B, DEC1A, DEC1B };
constexpr int kHeadIn = 16, kHeadOut = 3, kInCh = 16;

int64_t layer_offset(int l)
{
    int64_t off = 0;
    for (int k = 0; k < l; ++k) off += 27LL * kConv[k].cin * kConv[k].cout + kConv[k].cout;
    return off;
}
int64_t head_offset() { return layer_offset(kLayers); }
int64_t total_params() { return head_offset() + kHeadIn * kHeadOut + kHeadOut; }

// ------------------------------------------------------------------ device helpers

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld_pair(const bf16* p) { return __ldg(reinterpret_cast<const unsigned int*>(p)); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t pack_raw(bf16 lo, bf16 hi)
{
    __nv_bfloat162 v;
    v.x = lo;
    v.y = hi;
    return *reinterpret_cast<const uint32_t*>(&v);
}

struct Dims {
    int nx, ny, nz, nvox, batch;
};

// Voxel v split into (batch, x, y, z) once, and shifted by (dx, dy, dz):
// periodic in x, y; -1 outside in z (a kernel shifts one voxel by up to 27
// taps).
struct VoxCoord {
    int b, x, y, z;  // b < 0: no voxel
};
__device__ __forceinline__ VoxCoord vox_coord(const Dims& d, int v)
{
    VoxCoord c{-1, 0, 0, 0};
    if (v < 0 || v >= d.nvox * d.batch) return c;
    c.b = v / d.nvox;
    const int r = v - c.b * d.nvox;
    c.x = r % d.nx;
    const int t = r / d.nx;
    c.y = t % d.ny;
    c.z = t / d.ny;
    return c;
}
__device__ __forceinline__ int shifted(const Dims& d, const VoxCoord& c, int dx, int dy, int dz)
{
    const int zs = c.z + dz;
    if (c.b < 0 || zs < 0 || zs >= d.nz) return -1;
    int xs = c.x + dx, ys = c.y + dy;
    xs = xs < 0 ? xs + d.nx : (xs >= d.nx ? xs - d.nx : xs);
    ys = ys < 0 ? ys + d.ny : (ys >= d.ny ? ys - d.ny : ys);
    return c.b * d.nvox + xs + d.nx * (ys + d.ny * zs);
}

// ------------------------------------------------------------------ convolution: forward

struct ConvFwd {
    const bf16* src1;
    int c1;
    const bf16* src2;  // concatenated after src1 (may be null, c2 = 0)
    int c2;
    const bf16* w;     // [27][cout][cin]
    const float* bias; // [cout]
    bf16* dst;         // [vox][cout]
    Dims d;
    int relu;
    int* status;       // set to 1 when a bounded wait of the tensor-core kernel expires
    int tps;           // taps per shared-memory stage of the tensor-core kernel (1..9)
};

// ------------------------------------------------------------------ convolution: forward on tcgen05
//
// One CTA (four warps) computes 128 output voxels x COUT channels, the
// implicit GEMM D[128][COUT] = sum over the 27 taps of A_t[128][cin] W_t^T,
// A_t the cin input channels of the tap-shifted voxels.  Per tap, A_t and W_t
// are copied into shared memory with 16-byte cp.async (zero rows where the tap
// leaves the volume in z) in the tensor core's no-swizzle K-major layout:
// core matrices of 8 rows x 16 bytes, adjacent core matrices along K 128 bytes
// apart (LBO), along M / N cin/8 x 128 bytes apart (SBO).  A stage holds tps
// consecutive taps (tc_taps_per_stage: as many as fit in 14 KB, 1 to 9);
// one thread issues their cin/16 MMAs each (tcgen05.mma kind::f16, BF16 x
// BF16 -> FP32, M = 128, N = COUT, K = 16) into a TMEM accumulator and commits
// them to the stage's mbarrier; two stages let the copies of the next taps
// overlap the MMAs of these.  The epilogue reads each warp's 32 accumulator rows with
// tcgen05.ld, adds the bias, applies the ReLU and stores BF16 rows.  Every
// mbarrier wait is bounded: on expiry the kernel raises a.status, skips the
// epilogue, waits for its copies and frees its TMEM.

constexpr int kTcM = 128;
constexpr int kTcThreads = 128;
constexpr int kTcMaxCin = 96;
constexpr int kTcMaxCout = 64;
// A stage holds as many taps as fit in kTcStageBytes (at least one, at most 9:
// one dz plane of the stencil), so that thin layers commit a K of several
// taps per barrier round trip while several CTAs still fit on an SM.
constexpr size_t kTcStageBytes = 14 * 1024;
constexpr size_t kTcWidestTap = (size_t)(kTcM + kTcMaxCout) * kTcMaxCin * sizeof(bf16);
constexpr size_t kTcSmem = 2 * (kTcWidestTap > kTcStageBytes ? kTcWidestTap : kTcStageBytes) + 64;
inline int tc_taps_per_stage(int cin, int cout)
{
    const size_t tap = (size_t)(kTcM + cout) * cin * sizeof(bf16);
    const int t = (int)(kTcStageBytes / tap);
    return t < 1 ? 1 : (t > 9 ? 9 : t);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor of the tensor core: no swizzle, start
// address, LBO and SBO in 16-byte units, descriptor version 1 (bits 46-48).
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 D (bits 4-5 = 1), BF16 A (7-9 = 1)
// and B (10-12 = 1), both K-major, N / 8 in bits 17-22, M / 16 in bits 24-28.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
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

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int COUT>
__global__ void __launch_bounds__(kTcThreads) conv_fwd_tc_kernel(const ConvFwd a)
{
    extern __shared__ __align__(128) unsigned char tc_smem[];
    const int cin = a.c1 + a.c2;
    const int kb = cin / 8;                        // 16-byte core-matrix columns along K
    const uint32_t sbo_a = (uint32_t)kb * 128u;    // between 8-row groups
    const uint32_t a_bytes = kTcM * cin * 2, b_bytes = COUT * cin * 2;
    const int tps = a.tps;                              // taps per stage
    const uint32_t tap_bytes = a_bytes + b_bytes, stage_bytes = (uint32_t)tps * tap_bytes;
    const int stages = (27 + tps - 1) / tps;
    const uint32_t smem0 = smem_u32(tc_smem);  // stage s starts at smem0 + s stage_bytes
    uint64_t* bars = reinterpret_cast<uint64_t*>(tc_smem + 2 * stage_bytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2);
    constexpr uint32_t kCols = COUT < 32 ? 32 : COUT;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int total = a.d.nvox * a.d.batch;
    const int v0 = blockIdx.x * kTcM;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bars[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bars[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    // Thread tid stages A row tid (voxel v0 + tid) for every tap: its
    // coordinates are split once here, and a tap only shifts and wraps them.
    static_assert(kTcM == kTcThreads, "one A row per thread");
    const VoxCoord row = vox_coord(a.d, v0 + tid);
    const uint32_t arow = (uint32_t)(tid >> 3) * sbo_a + (uint32_t)(tid & 7) * 16u;

    // copies of tap t into slot tt of stage s: the A rows (voxels) and the W_t rows (output channels)
    auto load_tap = [&](int t, int s, int tt) {
        const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
        const uint32_t sa = (smem0 + (uint32_t)s * stage_bytes) + (uint32_t)tt * tap_bytes, sb = sa + a_bytes;
        {
            const int sv = shifted(a.d, row, dx, dy, dz);  // -1 beyond the plates (zero fill)
            const bf16* s1 = sv >= 0 ? a.src1 + (size_t)sv * a.c1 : a.src1;
            const bf16* s2 = sv >= 0 ? a.src2 + (size_t)sv * a.c2 : a.src1;
            for (int q = 0; q < kb; ++q) {
                const int c = q * 8;
                cp_async16(sa + arow + (uint32_t)q * 128u, c < a.c1 ? s1 + c : s2 + (c - a.c1), sv >= 0);
            }
        }
        const bf16* w = a.w + (size_t)t * COUT * cin;
        for (int i = tid; i < COUT * kb; i += kTcThreads) {
            const int n = i / kb, q = i - n * kb;
            cp_async16(sb + (uint32_t)(n >> 3) * sbo_a + (uint32_t)q * 128u + (uint32_t)(n & 7) * 16u,
                       w + (size_t)n * cin + q * 8, true);
        }
    };
    // stage g: taps g tps .. g tps + tps - 1, one commit group
    auto load_stage = [&](int g, int s) {
        for (int tt = 0; tt < tps; ++tt) {
            const int t = g * tps + tt;
            if (t < 27) load_tap(t, s, tt);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    constexpr uint32_t idesc = umma_idesc_bf16(kTcM, COUT);
    bool ok = true;
    load_stage(0, 0);
    for (int g = 0; g < stages; ++g) {
        const int s = g & 1;
        if (g + 1 < stages) {
            if (g >= 1) ok = ok && mbar_wait(smem_u32(&bars[s ^ 1]), ((g - 1) >> 1) & 1);  // MMAs of stage g - 1
            if (ok) load_stage(g + 1, s ^ 1);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // the copies, to the tensor core's view
        ok = __syncthreads_and(ok) != 0;  // every thread takes the same branch
        if (!ok) break;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            for (int tt = 0; tt < tps && g * tps + tt < 27; ++tt) {
                const uint32_t sa = (smem0 + (uint32_t)s * stage_bytes) + (uint32_t)tt * tap_bytes, sb = sa + a_bytes;
                for (int j = 0; j < cin / 16; ++j) {
                    const uint64_t ad = umma_desc(sa + 256u * j, 128u, sbo_a);
                    const uint64_t bd = umma_desc(sb + 256u * j, 128u, sbo_a);
                    const uint32_t acc = (g > 0 || tt > 0 || j > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                        : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_u32(&bars[s]))
                         : "memory");
        }
    }
    // the commit of the last stage covers every MMA
    if (ok) ok = mbar_wait(smem_u32(&bars[(stages - 1) & 1]), ((stages - 1) >> 1) & 1);
    ok = __syncthreads_and(ok) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (ok) {
        const int r = warp * 32 + lane;
        const int v = v0 + r;
#pragma unroll
        for (int c0 = 0; c0 < COUT; c0 += 16) {
            float acc[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, acc);
            if (v < total) {
                uint32_t packed[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    float x0 = acc[2 * i] + a.bias[c0 + 2 * i], x1 = acc[2 * i + 1] + a.bias[c0 + 2 * i + 1];
                    if (a.relu) {
                        x0 = fmaxf(x0, 0.f);
                        x1 = fmaxf(x1, 0.f);
                    }
                    packed[i] = pack_bf16(x0, x1);
                }
                uint4* dst = reinterpret_cast<uint4*>(a.dst + (size_t)v * COUT + c0);
                dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
                dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
            }
        }
    } else if (tid == 0) {
        atomicExch(a.status, 1);
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kCols) : "memory");
    }
}

// ------------------------------------------------------------------ convolution: data gradient

struct ConvBwdData {
    const bf16* gp;     // [vox][cout] gradient of the pre-activation (ReLU mask applied), BF16
    const bf16* wt;     // [27][cin][cout] transposed weights
    float* dst1;        // [vox][c1] gradient of source 1 (overwritten)
    int c1;
    float* dst2;        // [vox][c2] gradient of source 2 (accumulated)
    int c2;
    int cout;
    Dims d;
};

template <int CIN>
__global__ void __launch_bounds__(128) conv_bwd_data_kernel(const ConvBwdData a)
{
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int tile = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int total = a.d.nvox * a.d.batch;
    const int v0 = tile * 16;
    if (v0 >= total) return;
    const int vA = v0 + g, vB = v0 + g + 8;
    const VoxCoord cA = vox_coord(a.d, vA), cB = vox_coord(a.d, vB);
    const int cout = a.cout;
    float acc[CIN / 8][4];
#pragma unroll
    for (int j = 0; j < CIN / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    for (int tap = 0; tap < 27; ++tap) {
        const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        // the output voxel that reads v through this tap sits at v - offset
        const int sA = shifted(a.d, cA, -dx, -dy, -dz);
        const int sB = shifted(a.d, cB, -dx, -dy, -dz);
        const bf16* wt = a.wt + (size_t)tap * CIN * cout;
        for (int c = 0; c < cout; c += 16) {
            uint32_t fa[4];
            const int cols[4] = {c + 2 * t, c + 2 * t, c + 8 + 2 * t, c + 8 + 2 * t};
            const int src[4] = {sA, sB, sA, sB};
#pragma unroll
            for (int q = 0; q < 4; ++q) fa[q] = src[q] >= 0 ? ld_pair(a.gp + (size_t)src[q] * cout + cols[q]) : 0u;
#pragma unroll
            for (int j = 0; j < CIN / 8; ++j) {
                const bf16* wr = wt + (size_t)(j * 8 + g) * cout + c;
                const uint32_t fb[2] = {ld_pair(wr + 2 * t), ld_pair(wr + 8 + 2 * t)};
                mma16816(acc[j], fa, fb);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < CIN / 8; ++j) {
        const int ci = j * 8 + 2 * t;
        const float r[4] = {acc[j][0], acc[j][1], acc[j][2], acc[j][3]};
        const int vv[2] = {vA, vB};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            for (int e = 0; e < 2; ++e) {
                const int cc = ci + e;
                const float val = r[2 * h + e];
                if (cc < a.c1)
                    a.dst1[(size_t)vv[h] * a.c1 + cc] = val;
                else
                    a.dst2[(size_t)vv[h] * a.c2 + (cc - a.c1)] += val;
            }
        }
    }
}

// ------------------------------------------------------------------ convolution: weight gradient

struct ConvBwdW {
    const bf16* gp;     // [vox][cout] gradient of the pre-activation (ReLU mask applied), BF16
    const bf16* src1;   // [vox][c1]
    int c1;
    const bf16* src2;   // [vox][c2]
    int c2;
    int cout;
    float* gw;          // [27][cout][cin] (accumulated)
    Dims d;
    int chunk;          // voxels per block
};

constexpr int kWChunkSub = 32;  // voxels staged per shared-memory round

// grid = (voxel chunks, 27 taps); 8 warps share the (cout/16) x (cin/8) tiles.
__global__ void __launch_bounds__(256) conv_bwd_w_kernel(const ConvBwdW a)
{
    extern __shared__ unsigned char smem_raw[];
    const int cin = a.c1 + a.c2;
    const int cout = a.cout;
    bf16* Gs = reinterpret_cast<bf16*>(smem_raw);  // [kWChunkSub][cout]
    bf16* Xs = Gs + kWChunkSub * cout;              // [kWChunkSub][cin]
    __shared__ int srow[kWChunkSub];                // tap-shifted source voxel of each staged row
    const int tap = blockIdx.y;
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    const int total = a.d.nvox * a.d.batch;
    const int vbeg = blockIdx.x * a.chunk;
    const int vend = min(vbeg + a.chunk, total);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int mt = cout / 16, nt = cin / 8, tiles = mt * nt;
    constexpr int kMaxTiles = 6;  // per warp: up to 48 tiles / 8 warps (cout 64 x cin 96 -> 4 x 12)
    float acc[kMaxTiles][4];
#pragma unroll
    for (int k = 0; k < kMaxTiles; ++k) acc[k][0] = acc[k][1] = acc[k][2] = acc[k][3] = 0.f;
    for (int s0 = vbeg; s0 < vend; s0 += kWChunkSub) {
        __syncthreads();
        if (threadIdx.x < kWChunkSub) {
            const int v = s0 + threadIdx.x;
            srow[threadIdx.x] = v < vend ? shifted(a.d, vox_coord(a.d, v), dx, dy, dz) : -1;
        }
        // 16-byte groups of 8 channels (cout, c1 and c2 are multiples of 8)
        const int cg = cout >> 3;
        for (int e = threadIdx.x; e < kWChunkSub * cg; e += blockDim.x) {
            const int r = e / cg, q = e - r * cg;
            const int v = s0 + r;
            uint4 gv = make_uint4(0u, 0u, 0u, 0u);
            if (v < vend) gv = __ldg(reinterpret_cast<const uint4*>(a.gp + (size_t)v * cout) + q);
            reinterpret_cast<uint4*>(Gs)[e] = gv;
        }
        __syncthreads();  // srow
        const int ig = cin >> 3, ig1 = a.c1 >> 3;
        for (int e = threadIdx.x; e < kWChunkSub * ig; e += blockDim.x) {
            const int r = e / ig, q = e - r * ig;
            const int sv = srow[r];
            uint4 xv = make_uint4(0u, 0u, 0u, 0u);
            if (sv >= 0)
                xv = q < ig1 ? __ldg(reinterpret_cast<const uint4*>(a.src1 + (size_t)sv * a.c1) + q)
                             : __ldg(reinterpret_cast<const uint4*>(a.src2 + (size_t)sv * a.c2) + (q - ig1));
            reinterpret_cast<uint4*>(Xs)[e] = xv;
        }
        __syncthreads();
        for (int kk = 0; kk < kWChunkSub; kk += 16) {
#pragma unroll
            for (int q = 0; q < kMaxTiles; ++q) {
                const int tile = warp + 8 * q;
                if (tile >= tiles) break;
                const int m0 = (tile / nt) * 16, n0 = (tile % nt) * 8;
                // A[co][v] = G[v][co]; B[v][ci] = X[v][ci]
                uint32_t fa[4], fb[2];
                fa[0] = pack_raw(Gs[(kk + 2 * t) * cout + m0 + g], Gs[(kk + 2 * t + 1) * cout + m0 + g]);
                fa[1] = pack_raw(Gs[(kk + 2 * t) * cout + m0 + g + 8], Gs[(kk + 2 * t + 1) * cout + m0 + g + 8]);
                fa[2] = pack_raw(Gs[(kk + 8 + 2 * t) * cout + m0 + g], Gs[(kk + 9 + 2 * t) * cout + m0 + g]);
                fa[3] = pack_raw(Gs[(kk + 8 + 2 * t) * cout + m0 + g + 8], Gs[(kk + 9 + 2 * t) * cout + m0 + g + 8]);
                fb[0] = pack_raw(Xs[(kk + 2 * t) * cin + n0 + g], Xs[(kk + 2 * t + 1) * cin + n0 + g]);
                fb[1] = pack_raw(Xs[(kk + 8 + 2 * t) * cin + n0 + g], Xs[(kk + 9 + 2 * t) * cin + n0 + g]);
                mma16816(acc[q], fa, fb);
            }
        }
    }
    float* gw = a.gw + (size_t)tap * cout * cin;
#pragma unroll
    for (int q = 0; q < kMaxTiles; ++q) {
        const int tile = warp + 8 * q;
        if (tile >= tiles) break;
        const int m0 = (tile / nt) * 16, n0 = (tile % nt) * 8;
        atomicAdd(&gw[(size_t)(m0 + g) * cin + n0 + 2 * t], acc[q][0]);
        atomicAdd(&gw[(size_t)(m0 + g) * cin + n0 + 2 * t + 1], acc[q][1]);
        atomicAdd(&gw[(size_t)(m0 + g + 8) * cin + n0 + 2 * t], acc[q][2]);
        atomicAdd(&gw[(size_t)(m0 + g + 8) * cin + n0 + 2 * t + 1], acc[q][3]);
    }
}

// Gradient of the pre-activation, once per layer: gp = BF16(gout masked by
// the ReLU, out > 0), the operand of both convolution gradients; and the
// bias gradient gb[co] += sum_v of the masked gout (FP32).  A thread takes
// 8-channel groups of voxels (32-byte gout loads, 16-byte stores); the grid
// stride is a multiple of cout/8, so a thread's group -- and its 8 bias
// partials -- stay fixed; the block sums them in shared memory and adds
// them to gb with one atomic per channel.
__global__ void __launch_bounds__(256) grad_prep_kernel(const float* __restrict__ gout, const bf16* __restrict__ out,
                                                        bf16* __restrict__ gp, float* gb, int cout, int total)
{
    __shared__ float bsum[64];
    const int cg = cout >> 3;
    for (int k = threadIdx.x; k < cout; k += blockDim.x) bsum[k] = 0.f;
    __syncthreads();
    const int64_t items = (int64_t)total * cg;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int q = (int)(i0 % cg);  // fixed: stride % cg == 0
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int64_t i = i0; i < items; i += stride) {
        const float4 g0 = __ldg(reinterpret_cast<const float4*>(gout) + 2 * i);
        const float4 g1 = __ldg(reinterpret_cast<const float4*>(gout) + 2 * i + 1);
        const uint4 y = __ldg(reinterpret_cast<const uint4*>(out) + i);
        const __nv_bfloat162* yh = reinterpret_cast<const __nv_bfloat162*>(&y);
        float g[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (!(__low2float(yh[k]) > 0.f)) g[2 * k] = 0.f;
            if (!(__high2float(yh[k]) > 0.f)) g[2 * k + 1] = 0.f;
        }
        uint4 o;
        o.x = pack_bf16(g[0], g[1]);
        o.y = pack_bf16(g[2], g[3]);
        o.z = pack_bf16(g[4], g[5]);
        o.w = pack_bf16(g[6], g[7]);
        reinterpret_cast<uint4*>(gp)[i] = o;
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += g[k];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) atomicAdd(&bsum[q * 8 + k], acc[k]);
    __syncthreads();
    for (int k = threadIdx.x; k < cout; k += blockDim.x) atomicAdd(&gb[k], bsum[k]);
}

// ------------------------------------------------------------------ pooling / upsampling

// dst (coarse) = mean of the 2x2x2 children in src (fine), channels-last, C channels
__global__ void pool_fwd_kernel(const bf16* __restrict__ src, bf16* __restrict__ dst, Dims fine, int C)
{
    const int cx = fine.nx / 2, cy = fine.ny / 2, cz = fine.nz / 2, cvox = cx * cy * cz;
    const int64_t total = (int64_t)cvox * fine.batch * C;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const int64_t v = i / C;
        const int b = (int)(v / cvox);
        const int r = (int)(v - (int64_t)b * cvox);
        const int x = r % cx, y = (r / cx) % cy, z = r / (cx * cy);
        float s = 0.f;
        for (int k = 0; k < 8; ++k) {
            const int fx = 2 * x + (k & 1), fy = 2 * y + ((k >> 1) & 1), fz = 2 * z + (k >> 2);
            s += __bfloat162float(src[((size_t)b * fine.nvox + fx + fine.nx * (fy + fine.ny * fz)) * C + c]);
        }
        dst[(size_t)v * C + c] = __float2bfloat16_rn(0.125f * s);
    }
}

// gsrc (fine) += gdst (coarse) / 8
__global__ void pool_bwd_kernel(const float* __restrict__ gdst, float* __restrict__ gsrc, Dims fine, int C)
{
    const int cx = fine.nx / 2, cy = fine.ny / 2;
    const int64_t total = (int64_t)fine.nvox * fine.batch * C;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const int64_t v = i / C;
        const int b = (int)(v / fine.nvox);
        const int r = (int)(v - (int64_t)b * fine.nvox);
        const int x = r % fine.nx, y = (r / fine.nx) % fine.ny, z = r / (fine.nx * fine.ny);
        const size_t cv = (size_t)b * (fine.nvox / 8) + x / 2 + cx * (y / 2 + cy * (z / 2));
        gsrc[i] += 0.125f * gdst[cv * C + c];
    }
}

// dst (fine) = src (coarse) nearest
__global__ void up_fwd_kernel(const bf16* __restrict__ src, bf16* __restrict__ dst, Dims fine, int C)
{
    const int cx = fine.nx / 2, cy = fine.ny / 2;
    const int64_t total = (int64_t)fine.nvox * fine.batch * C;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const int64_t v = i / C;
        const int b = (int)(v / fine.nvox);
        const int r = (int)(v - (int64_t)b * fine.nvox);
        const int x = r % fine.nx, y = (r / fine.nx) % fine.ny, z = r / (fine.nx * fine.ny);
        const size_t cv = (size_t)b * (fine.nvox / 8) + x / 2 + cx * (y / 2 + cy * (z / 2));
        dst[i] = src[cv * C + c];
    }
}

// gsrc (coarse) = sum of gdst over the 8 children (overwrites)
__global__ void up_bwd_kernel(const float* __restrict__ gdst, float* __restrict__ gsrc, Dims fine, int C)
{
    const int cx = fine.nx / 2, cy = fine.ny / 2, cz = fine.nz / 2, cvox = cx * cy * cz;
    const int64_t total = (int64_t)cvox * fine.batch * C;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const int64_t v = i / C;
        const int b = (int)(v / cvox);
        const int r = (int)(v - (int64_t)b * cvox);
        const int x = r % cx, y = (r / cx) % cy, z = r / (cx * cy);
        float s = 0.f;
        for (int k = 0; k < 8; ++k) {
            const int fx = 2 * x + (k & 1), fy = 2 * y + ((k >> 1) & 1), fz = 2 * z + (k >> 2);
            s += gdst[((size_t)b * fine.nvox + fx + fine.nx * (fy + fine.ny * fz)) * C + c];
        }
        gsrc[i] = s;
    }
}

// ------------------------------------------------------------------ input, head, loss, optimiser

// x[v][0..2] = n_ansatz, x[v][3] = q0 Lz / 2 pi, [4] = Lz / 32, [5] = W0 / 1e-3, rest 0.
__global__ void input_kernel(const float* __restrict__ n, const float* __restrict__ scal, bf16* __restrict__ x, Dims d)
{
    const int total = d.nvox * d.batch;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < total; v += gridDim.x * blockDim.x) {
        const int b = v / d.nvox, r = v - b * d.nvox;
        const float* nb = n + (size_t)b * 3 * d.nvox;
        float vals[kInCh];
        for (int c = 0; c < kInCh; ++c) vals[c] = 0.f;
        vals[0] = nb[r];
        vals[1] = nb[d.nvox + r];
        vals[2] = nb[2 * d.nvox + r];
        const float q0 = scal[3 * b], lz = scal[3 * b + 1], w0 = scal[3 * b + 2];
        vals[3] = q0 * lz / 6.283185307179586f;
        vals[4] = lz / 32.f;
        vals[5] = w0 / 1e-3f;
        uint32_t* dst = reinterpret_cast<uint32_t*>(x + (size_t)v * kInCh);
        for (int c = 0; c < kInCh; c += 2) dst[c / 2] = pack_bf16(vals[c], vals[c + 1]);
    }
}

// Head (1x1x1 conv 16 -> 3), residual on the ansatz, normalisation; optionally
// the loss mean |n - target|^2 and the gradients of d1, W_head, b_head.
__global__ void __launch_bounds__(256) head_kernel(const bf16* __restrict__ d1, const float* __restrict__ n_ans,
                                                   const float* __restrict__ params_head, float* __restrict__ n_out,
                                                   const float* __restrict__ target, float* __restrict__ g_d1,
                                                   float* __restrict__ g_head, float* __restrict__ loss, Dims d)
{
    __shared__ float sh[kHeadOut * kHeadIn + kHeadOut];
    __shared__ float red[kHeadOut * kHeadIn + kHeadOut + 1][8];
    for (int k = threadIdx.x; k < kHeadOut * kHeadIn + kHeadOut; k += blockDim.x) sh[k] = params_head[k];
    __syncthreads();
    const int total = d.nvox * d.batch;
    const float inv_total = 1.f / (float)total;
    float gacc[kHeadOut * kHeadIn + kHeadOut + 1];
    for (int k = 0; k < kHeadOut * kHeadIn + kHeadOut + 1; ++k) gacc[k] = 0.f;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < total; v += gridDim.x * blockDim.x) {
        const int b = v / d.nvox, r = v - b * d.nvox;
        float h[kHeadIn];
        for (int c = 0; c < kHeadIn; ++c) h[c] = __bfloat162float(d1[(size_t)v * kHeadIn + c]);
        float vv[3];
        for (int o = 0; o < 3; ++o) {
            float s = sh[kHeadOut * kHeadIn + o];
            for (int c = 0; c < kHeadIn; ++c) s += sh[o * kHeadIn + c] * h[c];
            vv[o] = n_ans[(size_t)b * 3 * d.nvox + o * d.nvox + r] + s;
        }
        const float len = sqrtf(vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2]);
        const float nn[3] = {vv[0] / len, vv[1] / len, vv[2] / len};
        if (n_out)
            for (int o = 0; o < 3; ++o) n_out[(size_t)b * 3 * d.nvox + o * d.nvox + r] = nn[o];
        if (target) {
            float gn[3], dot = 0.f, l = 0.f;
            for (int o = 0; o < 3; ++o) {
                const float diff = nn[o] - target[(size_t)b * 3 * d.nvox + o * d.nvox + r];
                l += diff * diff;
                gn[o] = 2.f * diff * inv_total;
                dot += gn[o] * nn[o];
            }
            gacc[kHeadOut * kHeadIn + kHeadOut] += l * inv_total;
            float gd[3];
            for (int o = 0; o < 3; ++o) gd[o] = (gn[o] - dot * nn[o]) / len;  // d/dv of v/|v|
            for (int c = 0; c < kHeadIn; ++c) {
                float s = 0.f;
                for (int o = 0; o < 3; ++o) {
                    s += sh[o * kHeadIn + c] * gd[o];
                    gacc[o * kHeadIn + c] += gd[o] * h[c];
                }
                g_d1[(size_t)v * kHeadIn + c] = s;
            }
            for (int o = 0; o < 3; ++o) gacc[kHeadOut * kHeadIn + o] += gd[o];
        }
    }
    if (!target) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < kHeadOut * kHeadIn + kHeadOut + 1; ++k) {
        float s = gacc[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[k][warp] = s;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kHeadOut * kHeadIn + kHeadOut + 1; k += blockDim.x) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[k][w];
        if (k < kHeadOut * kHeadIn + kHeadOut)
            atomicAdd(&g_head[k], s);
        else
            atomicAdd(loss, s);
    }
}

__global__ void bf16_to_f32_kernel(const bf16* __restrict__ a, float* __restrict__ out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __bfloat162float(a[i]);
}

__global__ void cast_params_kernel(const float* __restrict__ p, bf16* __restrict__ w, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        w[i] = __float2bfloat16_rn(p[i]);
}

// wt[tap][ci][co] = w[tap][co][ci]
__global__ void transpose_kernel(const float* __restrict__ p, bf16* __restrict__ wt, int cin, int cout)
{
    const int n = 27 * cin * cout;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int tap = i / (cin * cout);
        const int r = i - tap * cin * cout;
        const int ci = r / cout, co = r - ci * cout;
        wt[i] = __float2bfloat16_rn(p[(size_t)tap * cout * cin + (size_t)co * cin + ci]);
    }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

inline int grid_for(int64_t n, int threads = 256)
{
    int64_t b = (n + threads - 1) / threads;
    return (int)(b > 4096 ? 4096 : b);
}

}  // namespace

// ------------------------------------------------------------------ network runner

struct nh_unet {
    Dims lv[4];           // level dims (fine to coarse)
    int batch;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    size_t need = 0;
    // offsets into the workspace
    size_t wbf, wt[kLayers], x, act[kLayers], pool_[3], up_[3], grad_a, grad_b, grad_skip[3], gd1, gprep, status;
    std::string err;
};

namespace {

int unet_fail(nh_unet* u, int code, const std::string& m)
{
    if (u) u->err = m;
    nh::set_global_error(m);
    return code;
}

size_t al(size_t v) { return (v + 255) / 256 * 256; }

void plan(nh_unet* u)
{
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t o = off;
        off += al(b);
        return o;
    };
    const int64_t P = total_params();
    u->wbf = take(P * sizeof(bf16));
    for (int l = 0; l < kLayers; ++l) u->wt[l] = take(27 * (size_t)kConv[l].cin * kConv[l].cout * sizeof(bf16));
    const size_t V0 = (size_t)u->lv[0].nvox * u->batch;
    u->x = take(V0 * kInCh * sizeof(bf16));
    const int level_of[kLayers] = {0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0};
    for (int l = 0; l < kLayers; ++l)
        u->act[l] = take((size_t)u->lv[level_of[l]].nvox * u->batch * kConv[l].cout * sizeof(bf16));
    // pooled inputs of levels 1..3 and upsampled inputs of decoder levels 2..0
    const int pool_c[3] = {16, 16, 32};
    for (int k = 0; k < 3; ++k) u->pool_[k] = take((size_t)u->lv[k + 1].nvox * u->batch * pool_c[k] * sizeof(bf16));
    const int up_c[3] = {64, 32, 16};
    for (int k = 0; k < 3; ++k) u->up_[k] = take((size_t)u->lv[2 - k].nvox * u->batch * up_c[k] * sizeof(bf16));
    // gradient scratch: two ping-pong buffers large enough for any [vox][96] level-0..3 tensor,
    // three skip-gradient buffers (e1, e2, e3) and the head-input gradient
    size_t gmax = 0;
    for (int k = 0; k < 4; ++k) gmax = std::max(gmax, (size_t)u->lv[k].nvox * u->batch * 96);
    u->grad_a = take(gmax * sizeof(float));
    u->grad_b = take(gmax * sizeof(float));
    const int skip_c[3] = {16, 16, 32};
    for (int k = 0; k < 3; ++k) u->grad_skip[k] = take((size_t)u->lv[k].nvox * u->batch * skip_c[k] * sizeof(float));
    u->gd1 = take(V0 * kHeadIn * sizeof(float));
    size_t gp_max = 0;  // BF16 pre-activation gradient of the largest layer output
    for (int l = 0; l < kLayers; ++l)
        gp_max = std::max(gp_max, (size_t)u->lv[level_of[l]].nvox * u->batch * kConv[l].cout);
    u->gprep = take(gp_max * sizeof(bf16));
    u->status = take(sizeof(int));  // raised by an expired wait of the tensor-core convolution
    u->need = off;
}

template <typename T>
T* P(nh_unet* u, size_t off)
{
    return reinterpret_cast<T*>(u->ws + off);
}

cudaError_t conv_fwd(nh_unet* u, int l, int level, const bf16* s1, int c1, const bf16* s2, int c2,
                     const float* params, cudaStream_t st)
{
    ConvFwd a;
    a.src1 = s1;
    a.c1 = c1;
    a.src2 = s2;
    a.c2 = c2;
    a.w = P<bf16>(u, u->wbf) + layer_offset(l);
    a.bias = params + layer_offset(l) + 27LL * kConv[l].cin * kConv[l].cout;
    a.dst = P<bf16>(u, u->act[l]);
    a.d = u->lv[level];
    a.relu = 1;
    a.status = P<int>(u, u->status);
    static bool attr_set = false;  // the opt-in to more than 48 KB of shared memory, once per process
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(conv_fwd_tc_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kTcSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(conv_fwd_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(conv_fwd_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int cin = c1 + c2;
    if (cin % 16 || cin > kTcMaxCin || kConv[l].cout > kTcMaxCout) return cudaErrorInvalidValue;
    const int blocks = (a.d.nvox * a.d.batch + kTcM - 1) / kTcM;
    a.tps = tc_taps_per_stage(cin, kConv[l].cout);
    const size_t smem = 2 * (size_t)a.tps * (kTcM + kConv[l].cout) * cin * sizeof(bf16) + 64;
    switch (kConv[l].cout) {
    case 16: conv_fwd_tc_kernel<16><<<blocks, kTcThreads, smem, st>>>(a); break;
    case 32: conv_fwd_tc_kernel<32><<<blocks, kTcThreads, smem, st>>>(a); break;
    default: conv_fwd_tc_kernel<64><<<blocks, kTcThreads, smem, st>>>(a); break;
    }
    return cudaGetLastError();
}

// Backward of conv layer l: gout (FP32 [vox][cout]) -> data gradient into
// dst1 (c1 channels, overwritten) and dst2 (c2, accumulated); weight and bias
// gradients accumulated into grad.
cudaError_t conv_bwd(nh_unet* u, int l, int level, const float* gout, const bf16* s1, int c1, const bf16* s2, int c2,
                     float* dst1, float* dst2, float* grad, bool need_data, cudaStream_t st)
{
    const Dims d = u->lv[level];
    const int total = d.nvox * d.batch;
    const int cout = kConv[l].cout, cin = kConv[l].cin;
    const bf16* out = P<bf16>(u, u->act[l]);
    bf16* gp = P<bf16>(u, u->gprep);
    grad_prep_kernel<<<std::min(4 * 152, grid_for(total * (cout / 8), 256)), 256, 0, st>>>(
        gout, out, gp, grad + layer_offset(l) + 27LL * cin * cout, cout, total);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ConvBwdW w;
    w.gp = gp;
    w.src1 = s1;
    w.c1 = c1;
    w.src2 = s2;
    w.c2 = c2;
    w.cout = cout;
    w.gw = grad + layer_offset(l);
    w.d = d;
    w.chunk = 1024;
    dim3 grid((total + w.chunk - 1) / w.chunk, 27);
    const size_t smem = (size_t)kWChunkSub * (cin + cout) * sizeof(bf16);
    conv_bwd_w_kernel<<<grid, 256, smem, st>>>(w);
    e = cudaGetLastError();
    if (e != cudaSuccess || !need_data) return e;
    ConvBwdData b;
    b.gp = gp;
    b.wt = P<bf16>(u, u->wt[l]);
    b.dst1 = dst1;
    b.c1 = c1;
    b.dst2 = dst2;
    b.c2 = c2;
    b.cout = cout;
    b.d = d;
    const int blocks = (total / 16 + 3) / 4;
    switch (cin) {
    case 16: conv_bwd_data_kernel<16><<<blocks, 128, 0, st>>>(b); break;
    case 32: conv_bwd_data_kernel<32><<<blocks, 128, 0, st>>>(b); break;
    case 48: conv_bwd_data_kernel<48><<<blocks, 128, 0, st>>>(b); break;
    case 64: conv_bwd_data_kernel<64><<<blocks, 128, 0, st>>>(b); break;
    default: conv_bwd_data_kernel<96><<<blocks, 128, 0, st>>>(b); break;
    }
    return cudaGetLastError();
}

}  // namespace

#define UNET_CUDA(u, ...)                                                                      \
    do {                                                                                       \
        cudaError_t e_ = (__VA_ARGS__);                                                        \
        if (e_ != cudaSuccess) return unet_fail((u), NH_ECUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_)); \
    } while (0)

extern "C" {

int64_t nh_unet_param_count(void) { return total_params(); }

int nh_unet_create(int batch, int nx, int ny, int nz, nh_unet** out)
{
    if (!out) return unet_fail(nullptr, NH_EINVAL, "out is NULL");
    *out = nullptr;
    if (batch < 1 || nx < 16 || ny < 16 || nz < 8 || nx % 8 || ny % 8 || nz % 8)
        return unet_fail(nullptr, NH_EINVAL, "batch >= 1; nx, ny multiples of 8 and >= 16; nz a multiple of 8");
    if ((int64_t)nx * ny * nz * batch * 96 > 2000000000LL) return unet_fail(nullptr, NH_EINVAL, "problem too large");
    nh_unet* u = new (std::nothrow) nh_unet();
    if (!u) return unet_fail(nullptr, NH_ENOMEM, "host allocation failed");
    u->batch = batch;
    for (int k = 0; k < 4; ++k) {
        const int s = 1 << k;
        u->lv[k] = Dims{nx / s, ny / s, nz / s, (nx / s) * (ny / s) * (nz / s), batch};
    }
    if ((u->lv[3].nvox * batch) % 16) {
        delete u;
        return unet_fail(nullptr, NH_EINVAL, "the coarsest level must hold a multiple of 16 voxels");
    }
    plan(u);
    *out = u;
    return NH_OK;
}

int nh_unet_workspace_bytes(const nh_unet* u, size_t* bytes)
{
    if (!u || !bytes) return unet_fail(nullptr, NH_EINVAL, "NULL argument");
    *bytes = u->need;
    return NH_OK;
}

int nh_unet_bind(nh_unet* u, void* ws, size_t bytes)
{
    if (!u || !ws) return unet_fail(u, NH_EINVAL, "NULL argument");
    if (reinterpret_cast<uintptr_t>(ws) % 256) return unet_fail(u, NH_EINVAL, "workspace must be 256-byte aligned");
    if (bytes < u->need) return unet_fail(u, NH_ENOMEM, "workspace too small: need " + std::to_string(u->need));
    u->ws = static_cast<char*>(ws);
    u->ws_bytes = bytes;
    UNET_CUDA(u, cudaMemset(u->ws + u->status, 0, sizeof(int)));
    return NH_OK;
}

int nh_unet_status(nh_unet* u, void* stream)
{
    if (!u || !u->ws) return unet_fail(u, NH_EINVAL, "unbound network");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int flag = 0;
    UNET_CUDA(u, cudaMemcpyAsync(&flag, u->ws + u->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    UNET_CUDA(u, cudaStreamSynchronize(st));
    if (flag) {
        UNET_CUDA(u, cudaMemsetAsync(u->ws + u->status, 0, sizeof(int), st));
        return unet_fail(u, NH_ETIMEOUT, "a tensor-core convolution gave up waiting for its MMAs");
    }
    return NH_OK;
}

int nh_unet_set_params(nh_unet* u, const float* params, void* stream)
{
    if (!u || !u->ws || !params) return unet_fail(u, NH_EINVAL, "unbound network or NULL params");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t n = total_params();
    cast_params_kernel<<<grid_for(n), 256, 0, st>>>(params, P<bf16>(u, u->wbf), n);
    UNET_CUDA(u, cudaGetLastError());
    for (int l = 0; l < kLayers; ++l) {
        transpose_kernel<<<grid_for(27LL * kConv[l].cin * kConv[l].cout), 256, 0, st>>>(
            params + layer_offset(l), P<bf16>(u, u->wt[l]), kConv[l].cin, kConv[l].cout);
        UNET_CUDA(u, cudaGetLastError());
    }
    return NH_OK;
}

int nh_unet_forward(nh_unet* u, const float* params, const float* n_ansatz, const float* scalars, float* n_out,
                    void* stream)
{
    if (!u || !u->ws || !params || !n_ansatz || !scalars) return unet_fail(u, NH_EINVAL, "NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Dims d0 = u->lv[0];
    input_kernel<<<grid_for((int64_t)d0.nvox * d0.batch), 256, 0, st>>>(n_ansatz, scalars, P<bf16>(u, u->x), d0);
    UNET_CUDA(u, cudaGetLastError());
    auto act = [&](int l) { return P<bf16>(u, u->act[l]); };
    auto pool = [&](int k) { return P<bf16>(u, u->pool_[k]); };
    auto upb = [&](int k) { return P<bf16>(u, u->up_[k]); };
    UNET_CUDA(u, conv_fwd(u, ENC1A, 0, P<bf16>(u, u->x), 16, nullptr, 0, params, st));
    UNET_CUDA(u, conv_fwd(u, ENC1B, 0, act(ENC1A), 16, nullptr, 0, params, st));
    pool_fwd_kernel<<<grid_for((int64_t)u->lv[1].nvox * u->batch * 16), 256, 0, st>>>(act(ENC1B), pool(0), u->lv[0], 16);
    UNET_CUDA(u, conv_fwd(u, ENC2A, 1, pool(0), 16, nullptr, 0, params, st));
    UNET_CUDA(u, conv_fwd(u, ENC2B, 1, act(ENC2A), 16, nullptr, 0, params, st));
    pool_fwd_kernel<<<grid_for((int64_t)u->lv[2].nvox * u->batch * 16), 256, 0, st>>>(act(ENC2B), pool(1), u->lv[1], 16);
    UNET_CUDA(u, conv_fwd(u, ENC3A, 2, pool(1), 16, nullptr, 0, params, st));
    UNET_CUDA(u, conv_fwd(u, ENC3B, 2, act(ENC3A), 32, nullptr, 0, params, st));
    pool_fwd_kernel<<<grid_for((int64_t)u->lv[3].nvox * u->batch * 32), 256, 0, st>>>(act(ENC3B), pool(2), u->lv[2], 32);
    UNET_CUDA(u, conv_fwd(u, BOTA, 3, pool(2), 32, nullptr, 0, params, st));
    UNET_CUDA(u, conv_fwd(u, BOTB, 3, act(BOTA), 64, nullptr, 0, params, st));
    up_fwd_kernel<<<grid_for((int64_t)u->lv[2].nvox * u->batch * 64), 256, 0, st>>>(act(BOTB), upb(0), u->lv[2], 64);
    UNET_CUDA(u, conv_fwd(u, DEC3A, 2, upb(0), 64, act(ENC3B), 32, params, st));
    UNET_CUDA(u, conv_fwd(u, DEC3B, 2, act(DEC3A), 32, nullptr, 0, params, st));
    up_fwd_kernel<<<grid_for((int64_t)u->lv[1].nvox * u->batch * 32), 256, 0, st>>>(act(DEC3B), upb(1), u->lv[1], 32);
    UNET_CUDA(u, conv_fwd(u, DEC2A, 1, upb(1), 32, act(ENC2B), 16, params, st));
    UNET_CUDA(u, conv_fwd(u, DEC2B, 1, act(DEC2A), 16, nullptr, 0, params, st));
    up_fwd_kernel<<<grid_for((int64_t)u->lv[0].nvox * u->batch * 16), 256, 0, st>>>(act(DEC2B), upb(2), u->lv[0], 16);
    UNET_CUDA(u, conv_fwd(u, DEC1A, 0, upb(2), 16, act(ENC1B), 16, params, st));
    UNET_CUDA(u, conv_fwd(u, DEC1B, 0, act(DEC1A), 16, nullptr, 0, params, st));
    head_kernel<<<grid_for((int64_t)d0.nvox * d0.batch), 256, 0, st>>>(act(DEC1B), n_ansatz, params + head_offset(), n_out,
                                                                        nullptr, nullptr, nullptr, nullptr, d0);
    UNET_CUDA(u, cudaGetLastError());
    return NH_OK;
}

int nh_unet_backward(nh_unet* u, const float* params, const float* n_ansatz, const float* target, float* grad,
                     float* loss, void* stream)
{
    if (!u || !u->ws || !params || !n_ansatz || !target || !grad || !loss)
        return unet_fail(u, NH_EINVAL, "NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Dims d0 = u->lv[0];
    UNET_CUDA(u, cudaMemsetAsync(grad, 0, total_params() * sizeof(float), st));
    UNET_CUDA(u, cudaMemsetAsync(loss, 0, sizeof(float), st));
    auto act = [&](int l) { return P<bf16>(u, u->act[l]); };
    auto pool = [&](int k) { return P<bf16>(u, u->pool_[k]); };
    auto upb = [&](int k) { return P<bf16>(u, u->up_[k]); };
    float* ga = P<float>(u, u->grad_a);
    float* gb = P<float>(u, u->grad_b);
    float* gskip[3] = {P<float>(u, u->grad_skip[0]), P<float>(u, u->grad_skip[1]), P<float>(u, u->grad_skip[2])};
    float* gd1 = P<float>(u, u->gd1);
    head_kernel<<<std::min(256, grid_for((int64_t)d0.nvox * d0.batch)), 256, 0, st>>>(
        act(DEC1B), n_ansatz, params + head_offset(), nullptr, target, gd1, grad + head_offset(), loss, d0);
    UNET_CUDA(u, cudaGetLastError());
    // decoder level 0: dec1b <- gd1, dec1a <- ga  (sources [up2 | e1])
    UNET_CUDA(u, conv_bwd(u, DEC1B, 0, gd1, act(DEC1A), 16, nullptr, 0, ga, nullptr, grad, true, st));
    UNET_CUDA(u, cudaMemsetAsync(gskip[0], 0, (size_t)d0.nvox * d0.batch * 16 * sizeof(float), st));
    UNET_CUDA(u, conv_bwd(u, DEC1A, 0, ga, upb(2), 16, act(ENC1B), 16, gb, gskip[0], grad, true, st));
    up_bwd_kernel<<<grid_for((int64_t)u->lv[1].nvox * u->batch * 16), 256, 0, st>>>(gb, ga, u->lv[0], 16);  // -> g(dec2b)
    UNET_CUDA(u, cudaGetLastError());
    // decoder level 1
    UNET_CUDA(u, conv_bwd(u, DEC2B, 1, ga, act(DEC2A), 16, nullptr, 0, gb, nullptr, grad, true, st));
    UNET_CUDA(u, cudaMemsetAsync(gskip[1], 0, (size_t)u->lv[1].nvox * u->batch * 16 * sizeof(float), st));
    UNET_CUDA(u, conv_bwd(u, DEC2A, 1, gb, upb(1), 32, act(ENC2B), 16, ga, gskip[1], grad, true, st));
    up_bwd_kernel<<<grid_for((int64_t)u->lv[2].nvox * u->batch * 32), 256, 0, st>>>(ga, gb, u->lv[1], 32);  // -> g(dec3b)
    UNET_CUDA(u, cudaGetLastError());
    // decoder level 2
    UNET_CUDA(u, conv_bwd(u, DEC3B, 2, gb, act(DEC3A), 32, nullptr, 0, ga, nullptr, grad, true, st));
    UNET_CUDA(u, cudaMemsetAsync(gskip[2], 0, (size_t)u->lv[2].nvox * u->batch * 32 * sizeof(float), st));
    UNET_CUDA(u, conv_bwd(u, DEC3A, 2, ga, upb(0), 64, act(ENC3B), 32, gb, gskip[2], grad, true, st));
    up_bwd_kernel<<<grid_for((int64_t)u->lv[3].nvox * u->batch * 64), 256, 0, st>>>(gb, ga, u->lv[2], 64);  // -> g(botb)
    UNET_CUDA(u, cudaGetLastError());
    // bottleneck
    UNET_CUDA(u, conv_bwd(u, BOTB, 3, ga, act(BOTA), 64, nullptr, 0, gb, nullptr, grad, true, st));
    UNET_CUDA(u, conv_bwd(u, BOTA, 3, gb, pool(2), 32, nullptr, 0, ga, nullptr, grad, true, st));   // ga = g(pool2 out)
    pool_bwd_kernel<<<grid_for((int64_t)u->lv[2].nvox * u->batch * 32), 256, 0, st>>>(ga, gskip[2], u->lv[2], 32);
    UNET_CUDA(u, cudaGetLastError());
    // encoder level 2 (e3 gradient complete in gskip[2])
    UNET_CUDA(u, conv_bwd(u, ENC3B, 2, gskip[2], act(ENC3A), 32, nullptr, 0, ga, nullptr, grad, true, st));
    UNET_CUDA(u, conv_bwd(u, ENC3A, 2, ga, pool(1), 16, nullptr, 0, gb, nullptr, grad, true, st));
    pool_bwd_kernel<<<grid_for((int64_t)u->lv[1].nvox * u->batch * 16), 256, 0, st>>>(gb, gskip[1], u->lv[1], 16);
    UNET_CUDA(u, cudaGetLastError());
    // encoder level 1
    UNET_CUDA(u, conv_bwd(u, ENC2B, 1, gskip[1], act(ENC2A), 16, nullptr, 0, ga, nullptr, grad, true, st));
    UNET_CUDA(u, conv_bwd(u, ENC2A, 1, ga, pool(0), 16, nullptr, 0, gb, nullptr, grad, true, st));
    pool_bwd_kernel<<<grid_for((int64_t)d0.nvox * d0.batch * 16), 256, 0, st>>>(gb, gskip[0], u->lv[0], 16);
    UNET_CUDA(u, cudaGetLastError());
    // encoder level 0 (the input needs no gradient)
    UNET_CUDA(u, conv_bwd(u, ENC1B, 0, gskip[0], act(ENC1A), 16, nullptr, 0, ga, nullptr, grad, true, st));
    UNET_CUDA(u, conv_bwd(u, ENC1A, 0, ga, P<bf16>(u, u->x), 16, nullptr, 0, nullptr, nullptr, grad, false, st));
    return NH_OK;
}

int nh_unet_activation(nh_unet* u, int layer, float* out, void* stream)
{
    if (!u || !u->ws || !out || layer < 0 || layer >= kLayers) return unet_fail(u, NH_EINVAL, "bad arguments");
    const int level_of[kLayers] = {0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0};
    const int64_t n = (int64_t)u->lv[level_of[layer]].nvox * u->batch * kConv[layer].cout;
    bf16_to_f32_kernel<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(P<bf16>(u, u->act[layer]), out, n);
    UNET_CUDA(u, cudaGetLastError());
    return NH_OK;
}

int nh_unet_adam(float* params, const float* grad, float* m, float* v, int64_t count, int step, float lr, void* stream)
{
    if (!params || !grad || !m || !v || count < 1 || step < 1) return unet_fail(nullptr, NH_EINVAL, "bad Adam arguments");
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<grid_for(count), 256, 0, static_cast<cudaStream_t>(stream)>>>(params, grad, m, v, count, lr, b1, b2,
                                                                                 1e-8f, c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return unet_fail(nullptr, NH_ECUDA, std::string("adam: ") + cudaGetErrorString(e));
    return NH_OK;
}

void nh_unet_destroy(nh_unet* u) { delete u; }

}  // extern "C"
