// Host-side TMA descriptor encoding (driver entry point fetched through the runtime).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace nslct {

namespace {
PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  });
  return fn;
}
}  // namespace

bool encode_column_map(CUtensorMap* map, const void* base, int Nx, int Ny, int P) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
  if (!enc) return false;
  const int rows = Nx / 2;
  const cuuint64_t dims[2] = {(cuuint64_t)(2 * Ny), (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(2 * Ny) * 8};
  const cuuint32_t box[2] = {(cuuint32_t)(2 * P), (cuuint32_t)(rows <= 256 ? rows : (rows % 256 == 0 ? 256 : 128))};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool encode_column_map_batched(CUtensorMap* map, const void* base, int Nx, int Ny, int P, int nbatch,
                               long long bstride, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
  if (!enc || nbatch < 1 || (nbatch > 1 && (bstride < (long long)Nx * Ny || (bstride & 1)))) return false;
  const int rows = Nx / 2;
  const cuuint64_t dims[3] = {(cuuint64_t)(2 * Ny), (cuuint64_t)rows, (cuuint64_t)nbatch};
  const cuuint64_t strides[2] = {(cuuint64_t)(2 * Ny) * 8, (cuuint64_t)(nbatch > 1 ? bstride : (long long)Nx * Ny) * 8};
  if (box_rows < 1 || box_rows > 256 || rows % box_rows) return false;
  const cuuint32_t box[3] = {(cuuint32_t)(2 * P), (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace nslct
