// Tensor-memory-accelerator (TMA) tile copies of the column passes.
//
// A column-pass block owns a panel of P adjacent columns of one plane's
// intermediate slot ([M][ldw] complex, row-major).  Its rows are only 8P
// bytes wide, so plain per-thread loads touch one L1 line per row; a TMA
// tile copy moves the whole [M][P] panel between the slot and shared
// memory in one instruction instead, off the L1 load/store pipe.  Each
// plane has a 3-D tensor map over its slot, viewed as FP32
// {2 ldw, R1, M / R1} with R1 the largest divisor of M up to 256, so one
// box {2P, R1, M / R1} is the whole panel.  The slot's base and pitch are
// multiples of 16 bytes (even c0al and ldw) and a panel starts at an even
// column, so x = 2 (column - c0al) is a multiple of 4 floats = 16 bytes.
// Boxes past the slot's last column read zeros and store nothing.
#pragma once

#include "ffst_internal.cuh"

namespace ffst {

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// Thread 0; the caller then passes a block barrier before any use.
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Thread 0: expect `bytes` on the barrier and start the panel load.
__device__ __forceinline__ void tma_load_panel(const CUtensorMap* map, float2* dst, uint64_t* bar, int x,
                                               unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(0), "r"(0), "r"(smem_u32(bar))
      : "memory");
}

// All threads: wait for the barrier's phase `parity` to complete, at most
// about a second; false (and *err |= 2) when it does not.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* err) {
  const unsigned a = smem_u32(bar);
  for (int it = 0; it < (1 << 22); ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (it > 64) __nanosleep(128);
  }
  if (err) atomicOr(err, 2);
  return false;
}

// Thread 0, after every thread's shared-memory writes of the panel and a
// proxy fence plus barrier: store the panel and wait until the copy has
// read shared memory (the buffer is reused or released afterwards).
__device__ __forceinline__ void tma_store_panel(const CUtensorMap* map, const float2* src, int x) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(0), "r"(0), "r"(smem_u32(src))
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace ffst
