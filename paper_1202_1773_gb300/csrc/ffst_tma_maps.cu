// Host side of the TMA panel copies: one 3-D tensor map per plane over the
// plane's intermediate slot in its group buffer (layout in ffst_tma.cuh).
// The encoder is a driver function, reached through the runtime's
// entry-point query so the library links against the runtime only.
#include <cudaTypedefs.h>

#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "ffst_internal.cuh"

namespace ffst {

static PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

// Column lengths whose passes use TMA panels: the square sizes with fused
// launches (powers of two 256..4096).  FFST_TMA=0 turns them off.
static bool tma_wanted(const ffst_plan_s* p) {
  const char* e = std::getenv("FFST_TMA");
  if (e && e[0] == '0') return false;
  const int M = p->M;
  return M >= 256 && M <= 4096 && (M & (M - 1)) == 0;
}

void tma_free(ffst_plan_s* p) {
  cudaFree(p->d_tmaps);
  cudaFree(p->d_tmaps_inv);
  p->d_tmaps = nullptr;
  p->d_tmaps_inv = nullptr;
}

// Maps of one direction's layout (groups, slot offsets); false when the
// encoder rejects one.
static bool encode_layout(const ffst_plan_s* p, const std::vector<Group>& groups, const std::vector<long long>& off,
                          std::vector<CUtensorMap>& maps) {
  auto encode = encoder();
  if (!encode) return false;
  const int M = p->M, P = cols_per_cta(M);
  const int R1 = M < 256 ? M : 256;  // M is a power of two here
  maps.assign(p->eta, CUtensorMap{});
  for (size_t g = 0; g < groups.size(); ++g) {
    float2* base = p->d_H + (g % 2) * p->h_elems;
    for (int i = groups[g].p0; i < groups[g].p1; ++i) {
      const PlaneDesc& d = p->planes[i];
      if (d.W == 0) continue;  // never touched
      const cuuint64_t dims[3] = {(cuuint64_t)2 * d.ldw, (cuuint64_t)R1, (cuuint64_t)(M / R1)};
      const cuuint64_t strides[2] = {(cuuint64_t)d.ldw * sizeof(float2), (cuuint64_t)d.ldw * sizeof(float2) * R1};
      const cuuint32_t box[3] = {(cuuint32_t)(2 * P), (cuuint32_t)R1, (cuuint32_t)(M / R1)};
      const cuuint32_t estr[3] = {1, 1, 1};
      const CUresult r = encode(&maps[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base + off[i], dims, strides, box, estr,
                                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return false;
    }
  }
  return true;
}

static cudaError_t upload(CUtensorMap** dst, const std::vector<CUtensorMap>& maps) {
  cudaError_t e = cudaMalloc(dst, maps.size() * sizeof(CUtensorMap));
  if (e == cudaSuccess) e = cudaMemcpy(*dst, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice);
  return e;
}

// (Re)build the maps of both directions for the current group buffers;
// leaves them null (plain loads and stores) when the size does not use TMA
// or the encoder rejects a map.
ffst_status tma_build(ffst_plan_s* p, const std::vector<long long>& off_fwd, const std::vector<long long>& off_inv) {
  tma_free(p);
  if (!tma_wanted(p) || !p->d_H) return FFST_OK;
  std::vector<CUtensorMap> mf, mi;
  if (!encode_layout(p, p->groups, off_fwd, mf) || !encode_layout(p, p->groups_inv, off_inv, mi)) return FFST_OK;
  cudaError_t e = upload(&p->d_tmaps, mf);
  if (e == cudaSuccess) e = upload(&p->d_tmaps_inv, mi);
  if (e != cudaSuccess) {
    tma_free(p);
    return cuda_fail(e, "tensor maps");
  }
  return FFST_OK;
}

}  // namespace ffst
