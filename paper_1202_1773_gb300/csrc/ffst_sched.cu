// Persistent, dependency-driven schedule of the plane passes (square images
// with a fused configuration, M = N in 256..4096).
//
// One launch per direction runs every plane pass of the transform.  The
// blocks (as many as fit on the GPU at once) take tasks from a queue built at
// plan time, in queue order, through one atomic counter:
//   forward:  column task = kSchedItems forward column items of one plane
//                 (2-column panels): G = psi_hat F, column IFFT, write the
//                 plane's intermediate;
//             row task    = kSchedRows row blocks (4 rows each) of one plane:
//                 row C2R, write the stack.
//   inverse:  row task    = kSchedRows row blocks of one coefficient plane:
//                 row R2C, write the plane's intermediate;
//             column task = one panel and one batch of consecutive planes:
//                 column FFTs, S += psi_hat * (that) on the support rows.
// The intermediates live in a ring buffer small enough to stay in L2.
// Dependencies are counters in device memory:
//   forward row task of plane p    waits for all column items of p;
//   forward column task of plane p waits for all row tasks of the planes
//                                  whose ring slots p's slot overlaps;
//   inverse column task (panel, b) waits for all row tasks of batch b and
//                                  for the panel's previous column task (the
//                                  S sums stay in plane order: deterministic);
//   inverse row task of plane p    waits for all column tasks of the batches
//                                  holding the planes p's slot overlaps.
// Every task waits only on tasks earlier in the queue, which running blocks
// have already taken, so the waits always end.  A wait that does not end
// within kSpinLimit polls (about a second) sets the plan's sticky error word, and
// every block then stops taking tasks; ffst_plan_check reports it.
#include <algorithm>
#include <cstdlib>
#include <vector>

#include "ffst_kernels.cuh"

namespace ffst {

constexpr long long kSpinLimit = 1LL << 23;  // polls of >= 100 ns: about a second

struct SchedArgs {
  const int4* tasks;
  int ntasks;
  int* ctl;        // [0] next task; counter arrays at the offsets below
  int off_cols, off_rows, off_batch, off_panel;
  int* err;        // sticky error word
  const int4* pdep;
  const int2* batch;
  const int* batch_tasks;
  const int* batch_part;  // per inverse batch: its partial accumulator
  int rbx;         // row tasks per plane
  float target;    // per-plane scale target of low-precision storage (0: FP32 stack)
  float* scale_out;  // per-plane scales written by the forward (low-precision storage)
  int stuck;       // test mode: the first task waits on a counter nothing increments
};

#ifndef FFST_SCHED_ROWS
#define FFST_SCHED_ROWS 4
#endif
#ifndef FFST_SCHED_ITEMS
#define FFST_SCHED_ITEMS 2
#endif
// Work per task: row blocks (kThreads/T rows each) of a row task, forward
// column items of a column task.  Bigger tasks spread the per-task
// bookkeeping (task fetch, dependency check, completion signal) over more work.
constexpr int kSchedRows = FFST_SCHED_ROWS;
constexpr int kSchedItems = FFST_SCHED_ITEMS;

__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0: poll until *ctr >= target, then an acquire fence.  False on
// timeout (sets *err) or when another block has reported an error.
__device__ bool wait_geq(const int* ctr, int target, int* err) {
  if (ld_relaxed(ctr) < target) {
    long long it = 0;
    for (; it < kSpinLimit; ++it) {
      __nanosleep(100);
      if (ld_relaxed(ctr) >= target) break;
      if ((it & 255) == 0 && ld_relaxed(err) != 0) return false;
    }
    if (it == kSpinLimit) {
      atomicOr(err, 1);
      return false;
    }
  }
  __threadfence();
  return true;
}

// Thread 0: add n to a counter after the whole block's writes (the caller
// has passed a __syncthreads since the last write).
__device__ __forceinline__ void signal(int* ctr, int n) {
  __threadfence();
  atomicAdd(ctr, n);
}

// Task queue walk shared by both kernels.  Thread 0 takes the next index
// while the block works on the current task, so the atomic's round trip is
// off the critical path.
struct TaskCursor {
  int next;  // thread 0 only: index taken for the following task
  __device__ __forceinline__ void start(const SchedArgs& s) {
    if (threadIdx.x == 0) next = atomicAdd(&s.ctl[0], 1);
  }
  __device__ __forceinline__ int take(const SchedArgs& s, int* slot) {
    __syncthreads();  // the previous task's reads of *slot and of shared memory are done
    if (threadIdx.x == 0) {
      *slot = next;
      if (next < s.ntasks) next = atomicAdd(&s.ctl[0], 1);
    }
    __syncthreads();
    return *slot;
  }
};

template <int M>
__global__ void __launch_bounds__(kThreads, FFST_MIN_BLOCKS)
    k_fwd_sched(SchedArgs s, FwdColsArgs ca, C2RArgs ra) {
  extern __shared__ __align__(128) float2 smem[];
  __shared__ int slot, ok;
  __shared__ float pscale;
  TaskCursor cur;
  cur.start(s);
  for (;;) {
    const int ti = cur.take(s, &slot);
    if (ti >= s.ntasks) return;
    const int4 task = s.tasks[ti];
    if (task.x == 0) {  // task.w column items from task.y, of plane task.z
      if (threadIdx.x == 0) {
        const int4 dep = s.pdep[task.z];
        bool good = !(s.stuck && ti == 0) || wait_geq(&s.ctl[1], 1, s.err);
        for (int q = dep.x; q <= dep.y && good; ++q) good = wait_geq(&s.ctl[s.off_rows + q], s.rbx, s.err);
        ok = good;
      }
      __syncthreads();
      if (!ok) return;
      for (int i = 0; i < task.w; ++i) fwd_cols_body<M>(ca, task.y + i, smem);
      __syncthreads();
      if (threadIdx.x == 0) signal(&s.ctl[s.off_cols + task.z], task.w);
    } else {  // task.w row blocks from task.z, of plane task.y
      const int p = task.y;
      if (threadIdx.x == 0) {
        const PlaneDesc d = ca.planes[p];
        ok = wait_geq(&s.ctl[s.off_cols + p], d.nitems, s.err);
        float sc = 1.0f;
        if (ok && s.target > 0.0f) {
          sc = plane_scale_of(ca.partials, d.item0, d.nitems, s.target);
          if (task.z == 0) s.scale_out[p] = sc;
        }
        pscale = sc;
      }
      __syncthreads();
      if (!ok) return;
      for (int r = 0; r < task.w; ++r) {
        if (r) __syncthreads();
        rows_c2r_body<M / 2>(ra, task.z + r, p, smem, pscale);
      }
      __syncthreads();
      if (threadIdx.x == 0) signal(&s.ctl[s.off_rows + p], task.w);
    }
  }
}

template <int M>
__global__ void __launch_bounds__(kThreads, FFST_MIN_BLOCKS)
    k_inv_sched(SchedArgs s, R2CArgs ra, InvColsArgs ca) {
  extern __shared__ __align__(128) float2 smem[];
  __shared__ int slot, ok;
  TaskCursor cur;
  cur.start(s);
  for (;;) {
    const int ti = cur.take(s, &slot);
    if (ti >= s.ntasks) return;
    const int4 task = s.tasks[ti];
    if (task.x == 0) {  // task.w row blocks from task.z, of plane task.y
      const int p = task.y;
      if (threadIdx.x == 0) {
        const int4 dep = s.pdep[p];
        bool good = true;
        for (int b = dep.z; b <= dep.w && good; ++b)
          good = wait_geq(&s.ctl[s.off_batch + b], s.batch_tasks[b], s.err);
        ok = good;
      }
      __syncthreads();
      if (!ok) return;
      for (int r = 0; r < task.w; ++r) {
        if (r) __syncthreads();
        rows_r2c_body<M / 2>(ra, task.z + r, p, smem);
      }
      __syncthreads();
      if (threadIdx.x == 0) signal(&s.ctl[s.off_rows + p], task.w);
    } else {  // panel task.z of batch task.y, the panel's task number task.w
      const int b = task.y;
      const int2 pr = s.batch[b];
      if (threadIdx.x == 0) {
        bool good = wait_geq(&s.ctl[s.off_panel + task.z], task.w, s.err);
        for (int q = pr.x; q < pr.y && good; ++q) good = wait_geq(&s.ctl[s.off_rows + q], s.rbx, s.err);
        ok = good;
      }
      __syncthreads();
      if (!ok) return;
      inv_cols_body<M>(ca, task.z, pr.x, pr.y, ca.S + s.batch_part[b] * ca.sstride, smem);
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&s.ctl[s.off_panel + task.z], 1);
        atomicAdd(&s.ctl[s.off_batch + b], 1);
      }
    }
  }
}

template <int M>
struct SchedCfg {
  static constexpr size_t SMEM =
      RowCfg<M / 2>::SMEM > ColCfg<M>::SMEM ? RowCfg<M / 2>::SMEM : ColCfg<M>::SMEM;
};

template <int M>
static cudaError_t fwd_sched_M(const Sched& sc, const SchedArgs& s, const FwdColsArgs& ca, const C2RArgs& ra,
                               cudaStream_t st) {
  cudaError_t e = set_smem(k_fwd_sched<M>, SchedCfg<M>::SMEM);
  if (e != cudaSuccess) return e;
  k_fwd_sched<M><<<sc.blocks, kThreads, SchedCfg<M>::SMEM, st>>>(s, ca, ra);
  return cudaGetLastError();
}

template <int M>
static cudaError_t inv_sched_M(const Sched& sc, const SchedArgs& s, const R2CArgs& ra, const InvColsArgs& ca,
                               cudaStream_t st) {
  cudaError_t e = set_smem(k_inv_sched<M>, SchedCfg<M>::SMEM);
  if (e != cudaSuccess) return e;
  k_inv_sched<M><<<sc.blocks, kThreads, SchedCfg<M>::SMEM, st>>>(s, ra, ca);
  return cudaGetLastError();
}

#define FFST_DISPATCH_SCHED(M, CALL)        \
  switch (M) {                              \
    case 256: return CALL(256);             \
    case 512: return CALL(512);             \
    case 1024: return CALL(1024);           \
    case 2048: return CALL(2048);           \
    case 4096: return CALL(4096);           \
    default: return cudaErrorNotSupported;  \
  }

// Resident blocks per SM of the persistent kernels (the smaller of the two).
template <int M>
static cudaError_t blocks_per_sm_M(int* n) {
  int a = 0, b = 0;
  cudaError_t e = set_smem(k_fwd_sched<M>, SchedCfg<M>::SMEM);
  if (e == cudaSuccess) e = set_smem(k_inv_sched<M>, SchedCfg<M>::SMEM);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_fwd_sched<M>, kThreads, SchedCfg<M>::SMEM);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_inv_sched<M>, kThreads, SchedCfg<M>::SMEM);
  *n = std::min(a, b);
  return e;
}

static cudaError_t sched_blocks_per_sm(int M, int* n) {
#define CALL_(MM) blocks_per_sm_M<MM>(n)
  FFST_DISPATCH_SCHED(M, CALL_)
#undef CALL_
}

static SchedArgs sched_args(const ffst_plan_s* p, bool fwd) {
  const Sched& sc = p->sched;
  SchedArgs s;
  s.tasks = fwd ? sc.d_fwd : sc.d_inv;
  s.ntasks = fwd ? sc.n_fwd : sc.n_inv;
  s.ctl = sc.d_ctl;
  s.off_cols = sc.off_cols;
  s.off_rows = sc.off_rows;
  s.off_batch = sc.off_batch;
  s.off_panel = sc.off_panel;
  s.err = p->d_err;
  s.pdep = sc.d_pdep;
  s.batch = sc.d_batch;
  s.batch_tasks = sc.d_batch_tasks;
  s.batch_part = sc.d_batch_part;
  s.rbx = sc.rbx;
  s.target = 0.0f;
  s.scale_out = nullptr;
  s.stuck = 0;
  return s;
}

cudaError_t launch_fwd_sched(const ffst_plan_s* p, FwdColsArgs ca, C2RArgs ra, float target, float* scale_out,
                             cudaStream_t st) {
  const Sched& sc = p->sched;
  cudaError_t e = cudaMemsetAsync(sc.d_ctl, 0, sizeof(int) * (size_t)sc.ctl_ints, st);
  if (e != cudaSuccess) return e;
  SchedArgs s = sched_args(p, true);
  s.target = scale_out ? target : 0.0f;
  s.scale_out = scale_out;
  s.stuck = p->sched_mode == 2;
  ca.planes = sc.d_planes;
  ca.items = p->d_items;
  ca.nitems = p->total_items;
  ca.H = sc.d_ring;
  ca.partials = scale_out ? p->d_partials : nullptr;
  ca.tmaps = nullptr;  // the maps describe the group buffers, not the ring
  ca.H_bytes = sc.ring_elems * (long long)sizeof(float2);
  ra.plane_scale = nullptr;  // the kernel passes the plane factor itself
  ra.src = sc.d_ring;
  ra.src_bytes = sc.ring_elems * (long long)sizeof(float2);
  ra.planes = sc.d_planes;
  ra.plane0 = 0;
#define CALL_(MM) fwd_sched_M<MM>(sc, s, ca, ra, st)
  FFST_DISPATCH_SCHED(p->M, CALL_)
#undef CALL_
}

cudaError_t launch_inv_sched(const ffst_plan_s* p, R2CArgs ra, InvColsArgs ca, cudaStream_t st) {
  const Sched& sc = p->sched;
  cudaError_t e = cudaMemsetAsync(sc.d_ctl, 0, sizeof(int) * (size_t)sc.ctl_ints, st);
  if (e != cudaSuccess) return e;
  const SchedArgs s = sched_args(p, false);
  ra.dst = sc.d_ring;
  ra.planes = sc.d_planes;
  ra.plane0 = 0;
  ca.H = sc.d_ring;
  ca.planes = sc.d_planes;
  ca.tmaps = nullptr;  // the maps describe the group buffers, not the ring
  ra.dst_bytes = sc.ring_elems * (long long)sizeof(float2);
  ca.H_bytes = sc.ring_elems * (long long)sizeof(float2);
#define CALL_(MM) inv_sched_M<MM>(sc, s, ra, ca, st)
  FFST_DISPATCH_SCHED(p->M, CALL_)
#undef CALL_
}

// ---------------------------------------------------------------------------
// plan-time construction
// ---------------------------------------------------------------------------

// Ring size of the intermediates.  The columns run two block windows ahead
// of the rows, and the ring must hold what lies in between or the tasks
// wait on ring reuse: at 2048x2048 J=5, fwd+inv took 6.3 ms with 64 MB,
// 3.6 ms with 128 MB and 3.3 ms with 256 MB (grouped launches: 2.47 ms).
// FFST_RING_MB overrides the default.
double default_ring_mb() {
  double mb = 256.0;
  if (const char* e = std::getenv("FFST_RING_MB")) {
    const double v = std::atof(e);
    if (v > 0.0) mb = v;
  }
  return mb;
}

void sched_free(ffst_plan_s* p) {
  Sched& sc = p->sched;
  cudaFree(sc.d_ring);
  cudaFree(sc.d_planes);
  cudaFree(sc.d_fwd);
  cudaFree(sc.d_inv);
  cudaFree(sc.d_pdep);
  cudaFree(sc.d_batch);
  cudaFree(sc.d_batch_tasks);
  cudaFree(sc.d_batch_part);
  cudaFree(sc.d_ctl);
  sc = Sched{};
}

template <class T>
static cudaError_t upload(T** dst, const std::vector<T>& v) {
  *dst = nullptr;
  if (v.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc(dst, v.size() * sizeof(T));
  if (e == cudaSuccess) e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

ffst_status sched_build(ffst_plan_s* p, double ring_mb) {
  sched_free(p);
  if (!fused_supported(p->M, p->N)) return FFST_OK;
  Sched& sc = p->sched;
  const int eta = p->eta, M = p->M;
  const int P = cols_per_cta(M);
  const int teams = kThreads / (p->N / 2 / row_E(p->N / 2));  // rows per row task
  sc.rbx = (M + teams - 1) / teams;
  sc.npanels = (p->Hc + P - 1) / P;

  // ring slots, in plane order, wrapping to the start when a slot would not fit
  long long ring = (long long)(ring_mb * 1024.0 * 1024.0 / sizeof(float2));
  long long biggest = 0;
  for (int i = 0; i < eta; ++i) biggest = std::max(biggest, (long long)M * p->planes[i].ldw);
  ring = std::max(ring, biggest);
  std::vector<PlaneDesc> rp = p->planes;
  std::vector<long long> lo(eta), hi(eta);
  long long cursor = 0;
  for (int i = 0; i < eta; ++i) {
    const long long n = (long long)M * rp[i].ldw;
    if (cursor + n > ring) cursor = 0;
    rp[i].off = n ? cursor : 0;
    lo[i] = cursor;
    hi[i] = cursor + n;
    cursor += n;
  }
  // ring predecessors: earlier planes whose slot overlaps (range [x, y])
  std::vector<int4> pdep(eta, make_int4(1, 0, 1, 0));
  for (int i = 0; i < eta; ++i) {
    if (hi[i] == lo[i]) continue;
    for (int q = 0; q < i; ++q)
      if (hi[q] > lo[q] && lo[q] < hi[i] && lo[i] < hi[q]) {
        if (pdep[i].x > pdep[i].y) pdep[i].x = q;
        pdep[i].y = q;
      }
  }
  // inverse batches: consecutive planes with at most a third of the ring
  // each, all summed into the same partial accumulator as in the grouped
  // launches (so both schedules add the same terms in the same order)
  std::vector<int2> batch;
  std::vector<int> batch_of(eta), batch_part;
  {
    long long acc = 0;
    int b0 = 0;
    for (int i = 0; i < eta; ++i) {
      const long long n = (long long)M * rp[i].ldw;
      if (i > b0 && (acc + n > ring / 3 || inv_part(p, i) != inv_part(p, b0))) {
        batch.push_back(make_int2(b0, i));
        batch_part.push_back(inv_part(p, b0));
        b0 = i;
        acc = 0;
      }
      acc += n;
      batch_of[i] = (int)batch.size();
    }
    batch.push_back(make_int2(b0, eta));
    batch_part.push_back(inv_part(p, b0));
  }
  sc.nbatch = (int)batch.size();
  for (int i = 0; i < eta; ++i)
    if (pdep[i].x <= pdep[i].y) {
      pdep[i].z = batch_of[pdep[i].x];
      pdep[i].w = batch_of[pdep[i].y];
    }
  // panels of each batch, and each panel's running task number
  std::vector<std::vector<int>> bpanels(sc.nbatch);
  for (int b = 0; b < sc.nbatch; ++b) {
    std::vector<char> hit(sc.npanels, 0);
    for (int q = batch[b].x; q < batch[b].y; ++q)
      if (rp[q].W > 0)
        for (int c = rp[q].c0 / P; c <= (rp[q].c0 + rp[q].W - 1) / P; ++c) hit[c] = 1;
    for (int c = 0; c < sc.npanels; ++c)
      if (hit[c]) bpanels[b].push_back(c);
  }
  std::vector<int> batch_tasks(sc.nbatch);
  for (int b = 0; b < sc.nbatch; ++b) batch_tasks[b] = (int)bpanels[b].size();

  {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = 0;
    const cudaError_t e = sched_blocks_per_sm(M, &per_sm);
    if (e != cudaSuccess) return cuda_fail(e, "persistent schedule occupancy");
    sc.blocks = sms * std::max(per_sm, 1);
  }
  // queue distance between a task and what it waits for: two windows of
  // resident blocks (0.5 and 1 window measured slower at 2048x2048 J=5)
  const long long lag = 2LL * sc.blocks;

  // forward queue: columns lead; rows of a plane follow its columns by `lag`
  std::vector<int4> fq;
  {
    const long long total_col = p->total_items, total_row = (long long)eta * sc.rbx;
    fq.reserve(total_col + total_row);
    std::vector<long long> col_end(eta, -1), row_end(eta, -1);
    int pc = 0, ic = 0, pr = 0, rr = 0;
    long long nc = 0, nr = 0;
    auto skip_empty = [&] {
      while (pc < eta && ic >= p->planes[pc].nitems) {
        col_end[pc] = (long long)fq.size();
        ++pc;
        ic = 0;
      }
    };
    skip_empty();
    while (nc + nr < total_col + total_row) {
      const long long pos = (long long)fq.size();
      bool col_hard = pc < eta, col_soft = col_hard;
      if (col_hard)
        for (int q = pdep[pc].x; q <= pdep[pc].y; ++q) {
          if (row_end[q] < 0) col_hard = col_soft = false;
          else if (pos - row_end[q] < lag) col_soft = false;
        }
      const bool row_hard = pr < eta && col_end[pr] >= 0;
      const bool row_soft = row_hard && pos - col_end[pr] >= lag;
      const double fc = total_col ? (double)nc / total_col : 1.0, fr = (double)nr / total_row;
      bool take_col;
      if (col_soft && (!row_soft || fc <= fr)) take_col = true;
      else if (row_soft) take_col = false;
      else if (row_hard) take_col = false;
      else if (col_hard) take_col = true;
      else return fail(FFST_ERR_INVALID_ARG, "forward schedule: no task can be placed");
      if (take_col) {
        const int n = std::min(kSchedItems, p->planes[pc].nitems - ic);
        fq.push_back(make_int4(0, p->planes[pc].item0 + ic, pc, n));
        ic += n;
        nc += n;
        skip_empty();
      } else {
        const int n = std::min(kSchedRows, sc.rbx - rr);
        fq.push_back(make_int4(1, pr, rr, n));
        nr += n;
        if ((rr += n) == sc.rbx) {
          row_end[pr] = (long long)fq.size();
          ++pr;
          rr = 0;
        }
      }
    }
  }
  // inverse queue: rows lead; a batch's column tasks follow its rows by `lag`
  std::vector<int4> iq;
  {
    long long total_col = 0;
    for (int b = 0; b < sc.nbatch; ++b) total_col += batch_tasks[b];
    const long long total_row = (long long)eta * sc.rbx;
    iq.reserve(total_col + total_row);
    std::vector<long long> row_end(eta, -1), batch_end(sc.nbatch, -1);
    std::vector<int> panel_count(sc.npanels, 0);
    int pr = 0, rr = 0, bc = 0, ic = 0;
    long long nc = 0, nr = 0;
    auto skip_empty = [&] {
      while (bc < sc.nbatch && ic >= batch_tasks[bc] && row_end[batch[bc].y - 1] >= 0) {
        batch_end[bc] = (long long)iq.size();
        ++bc;
        ic = 0;
      }
    };
    while (nc + nr < total_col + total_row) {
      skip_empty();
      const long long pos = (long long)iq.size();
      bool row_hard = pr < eta, row_soft = row_hard;
      if (row_hard)
        for (int b = pdep[pr].z; b <= pdep[pr].w; ++b) {
          if (batch_end[b] < 0) row_hard = row_soft = false;
          else if (pos - batch_end[b] < lag) row_soft = false;
        }
      const bool col_hard = bc < sc.nbatch && ic < batch_tasks[bc] && row_end[batch[bc].y - 1] >= 0;
      const bool col_soft = col_hard && pos - row_end[batch[bc].y - 1] >= lag;
      const double fc = total_col ? (double)nc / total_col : 1.0, fr = (double)nr / total_row;
      bool take_row;
      if (row_soft && (!col_soft || fr <= fc)) take_row = true;
      else if (col_soft) take_row = false;
      else if (col_hard) take_row = false;
      else if (row_hard) take_row = true;
      else return fail(FFST_ERR_INVALID_ARG, "inverse schedule: no task can be placed");
      if (take_row) {
        const int n = std::min(kSchedRows, sc.rbx - rr);
        iq.push_back(make_int4(0, pr, rr, n));
        nr += n;
        if ((rr += n) == sc.rbx) {
          row_end[pr] = (long long)iq.size();
          ++pr;
          rr = 0;
        }
      } else {
        const int panel = bpanels[bc][ic];
        iq.push_back(make_int4(1, bc, panel, panel_count[panel]++));
        ++ic;
        ++nc;
      }
    }
  }
  sc.n_fwd = (int)fq.size();
  sc.n_inv = (int)iq.size();

  // counters: [0] next task, [1] never incremented (test mode), then per
  // plane (columns, rows), per batch, per panel
  sc.off_cols = 32;
  sc.off_rows = sc.off_cols + eta;
  sc.off_batch = sc.off_rows + eta;
  sc.off_panel = sc.off_batch + sc.nbatch;
  sc.ctl_ints = sc.off_panel + sc.npanels;

  cudaError_t e = cudaMalloc(&sc.d_ring, sizeof(float2) * (size_t)ring);
  sc.ring_elems = ring;
  sc.ring_mb = ring_mb;
  if (e == cudaSuccess) e = upload(&sc.d_planes, rp);
  if (e == cudaSuccess) e = upload(&sc.d_fwd, fq);
  if (e == cudaSuccess) e = upload(&sc.d_inv, iq);
  if (e == cudaSuccess) e = upload(&sc.d_pdep, pdep);
  if (e == cudaSuccess) e = upload(&sc.d_batch, batch);
  if (e == cudaSuccess) e = upload(&sc.d_batch_tasks, batch_tasks);
  if (e == cudaSuccess) e = upload(&sc.d_batch_part, batch_part);
  if (e == cudaSuccess) e = cudaMalloc(&sc.d_ctl, sizeof(int) * (size_t)sc.ctl_ints);
  if (e != cudaSuccess) {
    sched_free(p);
    return cuda_fail(e, "persistent schedule");
  }
  sc.on = true;
  return FFST_OK;
}

}  // namespace ffst

using namespace ffst;

extern "C" ffst_status ffst_plan_schedule_info(ffst_plan_t plan, int* blocks, int* fwd_tasks, int* inv_tasks,
                                               double* ring_mb) {
  if (!plan) return fail(FFST_ERR_INVALID_ARG, "ffst_plan_schedule_info: plan is NULL");
  const Sched& sc = plan->sched;
  if (blocks) *blocks = sc.on ? sc.blocks : 0;
  if (fwd_tasks) *fwd_tasks = sc.on ? sc.n_fwd : 0;
  if (inv_tasks) *inv_tasks = sc.on ? sc.n_inv : 0;
  if (ring_mb) *ring_mb = sc.on ? (double)sc.ring_elems * sizeof(float2) / (1024.0 * 1024.0) : 0.0;
  return FFST_OK;
}
