// Fused launches for square images: one launch runs the column pass of one
// plane group together with the row pass of the previous group (forward),
// or the row pass of one group together with the column pass of the
// previous one (inverse).  The two halves touch different intermediate
// buffers, so they are independent and share the SMs.  The column blocks
// take the lowest block indices: they run longest (an inverse column block
// walks every plane of the group that meets its panel), and starting them
// first keeps them off the launch's tail (measured at 2048x2048 J=5:
// inverse 1.52 -> 1.34 ms, forward 1.31 -> 1.25 ms against interleaving the
// column blocks evenly among the row blocks).
#include "ffst_kernels.cuh"

namespace ffst {

template <int M>
struct FusedCfg {
  static constexpr size_t SMEM =
      RowCfg<M / 2>::SMEM > ColCfg<M>::SMEM ? RowCfg<M / 2>::SMEM : ColCfg<M>::SMEM;
};

template <int M>
__global__ void __launch_bounds__(kThreads, min_blocks_for(M)) k_fwd_fused(FwdColsArgs ca, int nc, C2RArgs ra, int rbx) {
  extern __shared__ __align__(128) float2 smem[];
  int ci = 0, ri = 0;
  if (split_cols_first(blockIdx.x, nc, &ci, &ri)) fwd_cols_body<M>(ca, ci, smem);
  else rows_c2r_body<M / 2>(ra, ri % rbx, ri / rbx, smem, c2r_plane_factor(ra, ri / rbx));
}

template <int M>
__global__ void __launch_bounds__(kThreads, min_blocks_for(M)) k_inv_fused(R2CArgs ra, int rbx, InvColsArgs ca, int nc) {
  extern __shared__ __align__(128) float2 smem[];
  int ci = 0, ri = 0;
  if (split_cols_first(blockIdx.x, nc, &ci, &ri)) {
    int q0, q1;
    float2* S;
    const int panel = inv_chunk(ca, ci, &q0, &q1, &S);
    inv_cols_body<M>(ca, panel, q0, q1, S, smem);
  } else {
    rows_r2c_body<M / 2>(ra, ri % rbx, ri / rbx, smem);
  }
}

template <int M>
static cudaError_t fwd_fused_M(const FwdColsArgs& ca, int nitems, const C2RArgs& ra, int nplanes, cudaStream_t s) {
  const int rbx = (ra.M + RowCfg<M / 2>::TEAMS - 1) / RowCfg<M / 2>::TEAMS;
  const int nr = rbx * nplanes;
  const int nc = nitems > 0 ? (nitems + kFwdItems - 1) / kFwdItems : 0;
  if (nc + nr == 0) return cudaSuccess;
  cudaError_t e = set_smem(k_fwd_fused<M>, FusedCfg<M>::SMEM);
  if (e != cudaSuccess) return e;
  FwdColsArgs cb = ca;
  cb.nitems = nitems;
  k_fwd_fused<M><<<nc + nr, kThreads, FusedCfg<M>::SMEM, s>>>(cb, nc, ra, rbx);
  return cudaGetLastError();
}

template <int M>
static cudaError_t inv_fused_M(const R2CArgs& ra, int nplanes, const InvColsArgs& ca, cudaStream_t s) {
  const int nc = ca.npanels * ca.nchunks;
  const int rbx = (ra.M + RowCfg<M / 2>::TEAMS - 1) / RowCfg<M / 2>::TEAMS;
  const int nr = rbx * nplanes;
  if (nc + nr == 0) return cudaSuccess;
  cudaError_t e = set_smem(k_inv_fused<M>, FusedCfg<M>::SMEM);
  if (e != cudaSuccess) return e;
  k_inv_fused<M><<<nc + nr, kThreads, FusedCfg<M>::SMEM, s>>>(ra, rbx, ca, nc);
  return cudaGetLastError();
}

bool fused_supported(int M, int N) { return M == N && M >= 256 && M <= 4096 && (M & (M - 1)) == 0; }

#define FFST_DISPATCH_FUSED(M, CALL)        \
  switch (M) {                              \
    case 256: return CALL(256);             \
    case 512: return CALL(512);             \
    case 1024: return CALL(1024);           \
    case 2048: return CALL(2048);           \
    case 4096: return CALL(4096);           \
    default: return cudaErrorNotSupported;  \
  }

cudaError_t launch_fwd_fused(int M, const FwdColsArgs& ca, int nitems, const C2RArgs& ra, int nplanes,
                             cudaStream_t s) {
#define CALL_(MM) fwd_fused_M<MM>(ca, nitems, ra, nplanes, s)
  FFST_DISPATCH_FUSED(M, CALL_)
#undef CALL_
}

cudaError_t launch_inv_fused(int M, const R2CArgs& ra, int nplanes, const InvColsArgs& ca, cudaStream_t s) {
#define CALL_(MM) inv_fused_M<MM>(ra, nplanes, ca, s)
  FFST_DISPATCH_FUSED(M, CALL_)
#undef CALL_
}

}  // namespace ffst
