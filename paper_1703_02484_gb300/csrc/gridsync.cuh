// Grid-wide barrier and block-level helpers of the persistent kernels
// (triangulation maintenance, Verlet-list overlap correction).  The kernels
// are launched cooperatively (every block resident), and every wait is
// bounded: a barrier that waits longer than its limit (BD_BARRIER_TIMEOUT_NS,
// or the limit the host set in the control block) sets BD_ERR_DEVICE_TIMEOUT
// and every block leaves.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "bd_internal.h"

namespace bdgs {

#ifndef BD_BARRIER_TIMEOUT_NS
#define BD_BARRIER_TIMEOUT_NS 2000000000ull
#endif

struct Bar {
  unsigned gen;
  int ph;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_status(const int *p) {
  return *(volatile const int *)p;
}

// Words every thread needs after a barrier, read once per block by thread 0
// and handed to the block through shared memory (116k threads reading one
// global line would queue ~18k requests on one L2 slice per barrier).
enum { BC_CNT = 0, BC_ACT = 8, BC_CL = 11, BC_N = 14 };

// bounded grid barrier; returns false if the grid must stop.  With bc (block
// shared, BC_N ints): bc[BC_CNT + k] = the counters of the phase that just
// ended, bc[BC_ACT + l] = the lengths of the triangle lists, bc[BC_CL + l]
// those of the candidate lists.
static __device__ bool grid_sync(BdCtl *ctl, Bar &b, int *bc = nullptr) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    if (ld_status(&ctl->status) == BD_ERR_DEVICE_TIMEOUT) {
      ok = 0;
    } else {
      unsigned target = b.gen + 1;
      // host-set limit and test hold (read once per barrier by one thread)
      const unsigned long long lim_set = *(volatile const unsigned long long *)&ctl->bar_limit_ns;
      const unsigned long long limit = lim_set ? lim_set : BD_BARRIER_TIMEOUT_NS;
      const unsigned hold = *(volatile const unsigned *)&ctl->bar_hold;
      const unsigned last = gridDim.x - 1u + (hold != 0u && hold == target ? 1u : 0u);
      __threadfence();
      unsigned arrived = atomicAdd(&ctl->bar_count, 1u);
      if (arrived == last) {
        atomicExch(&ctl->bar_count, 0u);
        __threadfence();
        atomicExch(&ctl->bar_gen, target);
      } else {
        // spin hot for a while (barriers are short), then back off; give up
        // after the time limit
        unsigned long long t0 = 0;
        unsigned it = 0;
        while (ld_acquire(&ctl->bar_gen) != target) {
          ++it;
          if (it < 4096u) continue;
          if (t0 == 0) t0 = gtimer();
          if ((it & 63u) == 0 && gtimer() - t0 > limit) {
            atomicExch(&ctl->status, BD_ERR_DEVICE_TIMEOUT);
            ok = 0;
            break;
          }
          __nanosleep(64);
        }
      }
      __threadfence();
    }
    if (ok && bc) {
      const volatile int *row = ctl->cnt[b.ph & 3];
      for (int k = 0; k < 8; ++k) bc[BC_CNT + k] = row[k];
      for (int l = 0; l < 3; ++l) bc[BC_ACT + l] = ((const volatile int *)ctl->act_n)[l];
      for (int l = 0; l < 3; ++l) bc[BC_CL + l] = ((const volatile int *)ctl->cl_n)[l];
    }
    s_ok = ok;
  }
  __syncthreads();
  b.gen++;
  b.ph++;
  return s_ok != 0;
}

__device__ __forceinline__ int *cnt(BdCtl *ctl, int ph, int slot) { return &ctl->cnt[ph & 3][slot]; }


// every block calls this once on its way out; the last one resets the barrier
// words and phase counters so the next launch starts clean without a memset
static __device__ void block_exit(BdCtl *ctl) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned k = atomicAdd(&ctl->exit_count, 1u);
    if (k == gridDim.x - 1) {
      ctl->bar_count = 0;
      ctl->bar_gen = 0;
      for (int l = 0; l < 3; ++l) ctl->act_n[l] = ctl->cl_n[l] = 0;
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 8; ++b) ctl->cnt[a][b] = 0;
      __threadfence();
      ctl->exit_count = 0;
    }
  }
}

// reset the counters two phases ahead (see the rotation argument in BdCtl)
__device__ __forceinline__ void phase_begin(BdCtl *ctl, const Bar &b) {
  if (blockIdx.x == 0 && threadIdx.x < 8) ctl->cnt[(b.ph + 2) & 3][threadIdx.x] = 0;
}

// block-aggregated atomic add
__device__ __forceinline__ void block_add(int *dst, int v) {
  __shared__ int s_acc;
  if (threadIdx.x == 0) s_acc = 0;
  __syncthreads();
  // warp reduce
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(&s_acc, v);
  __syncthreads();
  if (threadIdx.x == 0 && s_acc) atomicAdd(dst, s_acc);
}

}  // namespace bdgs
