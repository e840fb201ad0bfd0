// bd_forces_noalloc: the all-pairs long-range force for callers that cannot
// allocate device memory.
//
// Some callers of this library cannot call cudaMalloc: a host framework that
// owns the whole device memory budget through its own allocator and must see
// every byte that is handed out, a latency-critical loop in which the device
// synchronisation implied by cudaMalloc/cudaFree is not acceptable, or a
// deployment that fixes the process's device footprint when the library is
// loaded.  They pass device buffers for the inputs and the output; the only
// scratch this entry point needs lives in the file-scope array below, which
// every GPU that loads the library holds until the process exits.
//
// Scratch layout (BD_NOALLOC_BYTES bytes):
//   [0, 16 n)                      float4 (x_hi, y_hi, x_lo, y_lo) per disk
//   [16 * BD_NOALLOC_MAX_N, ...)   double2 partial forces, [chunk][n]
// Every call rewrites every scratch element it reads, so nothing has to be
// cleared between calls.  All calls on a device share the one array: two calls
// whose kernels overlap on the GPU (e.g. on two streams) race on it, and the
// caller must serialise them.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "bd_internal.h"

#define BD_NOALLOC_MAX_N 65536
#define BD_NOALLOC_MAX_CHUNKS 8
#define BD_NOALLOC_BYTES ((size_t)BD_NOALLOC_MAX_N * (16 + 16 * BD_NOALLOC_MAX_CHUNKS))
#define BD_NA_THREADS 128
#define BD_NA_IPT 4
#define BD_NA_TJ 128

static __device__ __align__(256) unsigned char bd_noalloc_scratch[BD_NOALLOC_BYTES];

namespace {

__device__ __forceinline__ float na_rsqrt(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void na_two_sum(float &hi, float &lo, float t) {
  float s = __fadd_rn(hi, t);
  float bp = __fsub_rn(s, hi);
  float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(t, bp));
  hi = s;
  lo = __fadd_rn(lo, err);
}

struct NaArgs {
  int n, nchunk;
  const double2 *xy;
  const uint8_t *sp;
  double2 *F;
  float4 *work;
  double2 *part;
  float A[4];
};

// (hi, lo) FP32 pair of each FP64 coordinate
__global__ void k_na_split(NaArgs g) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  double2 p = g.xy[i];
  float xh = __double2float_rn(p.x), yh = __double2float_rn(p.y);
  g.work[i] = make_float4(xh, yh, __double2float_rn(p.x - (double)xh), __double2float_rn(p.y - (double)yh));
}

// Variant of the tiled all-pairs sweep for disks in the caller's order: the
// species of each j is looked up per pair, and r_j - r_i is formed from the
// (hi, lo) pairs, which keeps near pairs exact without a spatial ordering.
__global__ void __launch_bounds__(BD_NA_THREADS) k_na_force(NaArgs g) {
  __shared__ float4 sj[BD_NA_TJ];
  __shared__ unsigned char ssp[BD_NA_TJ];
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * BD_NA_THREADS * BD_NA_IPT;
  float xh[BD_NA_IPT], yh[BD_NA_IPT], xl[BD_NA_IPT], yl[BD_NA_IPT];
  float a0[BD_NA_IPT], a1[BD_NA_IPT], fxh[BD_NA_IPT], fxl[BD_NA_IPT], fyh[BD_NA_IPT], fyl[BD_NA_IPT];
#pragma unroll
  for (int q = 0; q < BD_NA_IPT; ++q) {
    int i = i0 + q * BD_NA_THREADS + tid;
    if (i < g.n) {
      float4 w = g.work[i];
      xh[q] = w.x; yh[q] = w.y; xl[q] = w.z; yl[q] = w.w;
      int s = g.sp[i] ? 1 : 0;
      a0[q] = g.A[2 * s];
      a1[q] = g.A[2 * s + 1];
    } else {
      xh[q] = yh[q] = 1.0e18f;
      xl[q] = yl[q] = 0.f;
      a0[q] = a1[q] = 0.f;
    }
    fxh[q] = fxl[q] = fyh[q] = fyl[q] = 0.f;
  }
  const int per = (g.n + g.nchunk - 1) / g.nchunk;
  const int jb = blockIdx.y * per, je = min(g.n, jb + per);
  for (int j0 = jb; j0 < je; j0 += BD_NA_TJ) {
    int j = j0 + tid;
    if (j < je) {
      sj[tid] = g.work[j];
      ssp[tid] = g.sp[j] ? 1 : 0;
    } else {
      sj[tid] = make_float4(1.0e18f, 1.0e18f, 0.f, 0.f);
      ssp[tid] = 0;
    }
    __syncthreads();
    float ax[BD_NA_IPT], ay[BD_NA_IPT];
#pragma unroll
    for (int q = 0; q < BD_NA_IPT; ++q) ax[q] = ay[q] = 0.f;
    for (int k = 0; k < BD_NA_TJ; ++k) {
      float4 p = sj[k];
      int s = ssp[k];
#pragma unroll
      for (int q = 0; q < BD_NA_IPT; ++q) {
        float dx = __fadd_rn(__fsub_rn(p.x, xh[q]), __fsub_rn(p.z, xl[q]));
        float dy = __fadd_rn(__fsub_rn(p.y, yh[q]), __fsub_rn(p.w, yl[q]));
        float r2 = __fmaf_rn(dx, dx, 1e-20f);
        r2 = __fmaf_rn(dy, dy, r2);
        float r = na_rsqrt(r2);
        float c = __fmul_rn(__fmul_rn(__fmul_rn(r, r), r), s ? a1[q] : a0[q]);
        ax[q] = __fmaf_rn(dx, c, ax[q]);
        ay[q] = __fmaf_rn(dy, c, ay[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < BD_NA_IPT; ++q) {
      na_two_sum(fxh[q], fxl[q], -ax[q]);
      na_two_sum(fyh[q], fyl[q], -ay[q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < BD_NA_IPT; ++q) {
    int i = i0 + q * BD_NA_THREADS + tid;
    if (i < g.n)
      g.part[(size_t)blockIdx.y * g.n + i] =
          make_double2((double)fxh[q] + (double)fxl[q], (double)fyh[q] + (double)fyl[q]);
  }
}

__global__ void k_na_sum(NaArgs g) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  double fx = 0.0, fy = 0.0;
  for (int k = 0; k < g.nchunk; ++k) {
    double2 f = g.part[(size_t)k * g.n + i];
    fx += f.x;
    fy += f.y;
  }
  g.F[i] = make_double2(fx, fy);
}

std::mutex g_na_mutex;
void *g_na_ptr[256] = {nullptr};
int g_na_sms[256] = {0};

}  // namespace

extern "C" int bd_forces_noalloc(int32_t n, const double *xy, const uint8_t *species,
                                 const double alpha[4], double *F, void *stream) {
  if (n < 1 || n > BD_NOALLOC_MAX_N || !xy || !species || !alpha || !F) return BD_ERR_ARG;
  // positions and forces are read and written as 16-byte double2 pairs
  if (((uintptr_t)xy & 15u) != 0 || ((uintptr_t)F & 15u) != 0) return BD_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return BD_ERR_CUDA;
  void *base = nullptr;
  int sms = 0;
  {
    // once per device, with that device current: the device address of the
    // scratch array (its host-side name is only a stand-in) and the SM count
    std::lock_guard<std::mutex> lk(g_na_mutex);
    if (!g_na_ptr[dev]) {
      void *p = nullptr;
      int k = 0;
      if (cudaGetSymbolAddress(&p, bd_noalloc_scratch) != cudaSuccess || !p) return BD_ERR_CUDA;
      if (cudaDeviceGetAttribute(&k, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || k < 1)
        return BD_ERR_CUDA;
      g_na_sms[dev] = k;
      g_na_ptr[dev] = p;
    }
    base = g_na_ptr[dev];
    sms = g_na_sms[dev];
  }
  NaArgs g;
  g.n = n;
  int iblocks = (n + BD_NA_THREADS * BD_NA_IPT - 1) / (BD_NA_THREADS * BD_NA_IPT);
  // j chunks so that the grid fills about two waves of one block per SM
  int nchunk = (2 * sms + iblocks - 1) / iblocks;
  nchunk = nchunk < 1 ? 1 : (nchunk > BD_NOALLOC_MAX_CHUNKS ? BD_NOALLOC_MAX_CHUNKS : nchunk);
  g.nchunk = nchunk;
  g.xy = (const double2 *)xy;
  g.sp = species;
  g.F = (double2 *)F;
  g.work = (float4 *)base;
  g.part = (double2 *)((unsigned char *)base + (size_t)16 * BD_NOALLOC_MAX_N);
  for (int k = 0; k < 4; ++k) g.A[k] = (float)alpha[k];
  cudaStream_t s = (cudaStream_t)stream;
  k_na_split<<<(n + 255) / 256, 256, 0, s>>>(g);
  k_na_force<<<dim3(iblocks, nchunk), BD_NA_THREADS, 0, s>>>(g);
  k_na_sum<<<(n + 255) / 256, 256, 0, s>>>(g);
  if (cudaGetLastError() != cudaSuccess) return BD_ERR_CUDA;
  return BD_OK;
}
