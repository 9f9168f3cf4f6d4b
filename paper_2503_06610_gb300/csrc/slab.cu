// slab.cu -- halo rows of a channel split into slabs along y (the domain
// decomposition of a channel over several devices or contexts).
//
// A slab holds rows y0 - 1 .. y0 + ny_local of the global channel: its
// interior rows 1 .. ny_local and one ghost row on each side.  Every kernel
// runs over the whole slab, periodic in y within it, so the ghost rows come
// out wrong; before anything reads them they are overwritten with the
// neighbouring slab's interior rows:
//   - after every LB step, the populations that the interior pulls across
//     the face: the five with e_y = +1 into the lower ghost row and the five
//     with e_y = -1 into the upper one (Sec. II.C streaming);
//   - in an FD update, u before the predictor, n^P before the corrector, n
//     before the stress and sigma before the divergence (the radius-1
//     central differences of Sec. II.B).
// The copies are plain device copies between contexts on one device; the row
// list comes from slab_plan (api.cu), which the C ABI exports.
#include "nh_internal.cuh"

namespace nh {

namespace {

template <typename E>
__global__ void __launch_bounds__(256) row_copy_kernel(const RowCopyList list)
{
    const RowCopyItem& it = list.item[blockIdx.y];
    const E* __restrict__ src = static_cast<const E*>(it.src);
    E* __restrict__ dst = static_cast<E*>(it.dst);
    const int per_comp = it.nz * it.nx;
    const int total = it.comps * per_comp;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int c = i / per_comp;
        const int r = i - c * per_comp;
        const int z = r / it.nx;
        const int x = r - z * it.nx;
        dst[(size_t)c * it.dst_cstride + (size_t)z * it.dst_zstride + x] =
            src[(size_t)c * it.src_cstride + (size_t)z * it.src_zstride + x];
    }
}

}  // namespace

cudaError_t launch_row_copies(const RowCopyList& list, int elem_bytes, cudaStream_t st)
{
    if (list.count < 1) return cudaSuccess;
    if (list.count > kMaxRowCopies) return cudaErrorInvalidValue;
    int most = 0;
    for (int k = 0; k < list.count; ++k) most = max(most, list.item[k].comps * list.item[k].nz * list.item[k].nx);
    const dim3 grid((most + 255) / 256 < 64 ? (most + 255) / 256 : 64, list.count);
    switch (elem_bytes) {
    case 8: row_copy_kernel<unsigned long long><<<grid, 256, 0, st>>>(list); break;
    case 4: row_copy_kernel<unsigned int><<<grid, 256, 0, st>>>(list); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace nh
