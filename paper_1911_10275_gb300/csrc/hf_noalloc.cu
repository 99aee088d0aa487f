// hf_noalloc.cu - the one entry point of the library that allocates nothing.
//
// Some callers cannot call cudaMalloc at all: code running inside a memory
// pool or arena that owns every device byte of the process, code whose
// allocations are forbidden while a CUDA graph is being built around it, or
// embedded/real-time hosts that allocate only at start-up.  For them this
// file provides hf_increment_norms_noalloc: the four squared norms that decide
// Newton convergence (||dU||^2, ||U||^2, ||dP||^2, ||P||^2), computed from
// caller-owned device vectors.  It is a variant of the reduction inside
// hf_newton_step; instead of the handle's scratch it uses a fixed array in
// this library's device memory, so it needs no handle and no allocation.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/hf.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BLOCKS = 4096;                 // blocks of one call
constexpr int64_t NA_CHUNK = 64LL * NA_THREADS;     // unknowns per block
constexpr int64_t NA_MAX_N = NA_CHUNK * NA_MAX_BLOCKS;  // 67,108,864 unknowns

// Scratch shared by every call in the process: words [0, 4*NA_MAX_BLOCKS) hold
// 4 partial sums per block, word 4*NA_MAX_BLOCKS holds the ticket counter of
// the last-block reduction.  Every GPU that loads the library holds this
// array (128 KiB + 256 B) until the process exits.
constexpr int NA_TICKET = 4 * NA_MAX_BLOCKS;
constexpr int NA_WORDS = 4 * NA_MAX_BLOCKS + 32;
static __device__ __align__(256) double na_scratch[NA_WORDS];

constexpr int NA_MAX_DEVICES = 64;
std::mutex na_mutex;
double* na_ptr[NA_MAX_DEVICES] = {};

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Each block reduces one contiguous chunk; the last block to finish (ticket)
// adds the block partials in block order, so the result does not depend on
// scheduling.  The ticket is reset by the host before the launch.
__global__ void __launch_bounds__(NA_THREADS) k_increment_norms_noalloc(const double* __restrict__ dx,
                                                                        const double* __restrict__ x,
                                                                        int64_t n_u, int64_t n, double* out,
                                                                        double* sc) {
  __shared__ double sm[4][NA_THREADS / 32];
  __shared__ bool last;
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  int64_t lo = (int64_t)blockIdx.x * NA_CHUNK;
  int64_t hi = lo + NA_CHUNK < n ? lo + NA_CHUNK : n;
  for (int64_t i = lo + threadIdx.x; i < hi; i += NA_THREADS) {
    double d = dx[i], v = x[i];
    int p = i >= n_u ? 2 : 0;
    a[p] += d * d;
    a[p + 1] += v * v;
  }
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = 0; t < 4; ++t) {
    double s = na_warp_sum(a[t]);
    if (lane == 0) sm[t][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int w = 0; w < NA_THREADS / 32; ++w) s += sm[threadIdx.x][w];
    sc[blockIdx.x * 4 + threadIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(reinterpret_cast<unsigned int*>(sc + NA_TICKET), 1u) == gridDim.x - 1;
  __syncthreads();
  if (last && threadIdx.x < 4) {
    double s = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(&sc[b * 4 + threadIdx.x]);
    out[threadIdx.x] = s;
  }
}

void set_msg(char* err, int64_t err_len, const char* msg) {
  if (err && err_len > 0) snprintf(err, (size_t)err_len, "%s", msg);
}

}  // namespace

extern "C" hf_status hf_increment_norms_noalloc(const double* d_dx, const double* d_x, int64_t n_u, int64_t n_p,
                                                double* d_out, void* cuda_stream, char* err, int64_t err_len) {
  set_msg(err, err_len, "");
  if (!d_dx || !d_x || !d_out || n_u < 0 || n_p < 0) {
    set_msg(err, err_len, "hf_increment_norms_noalloc: null pointer or negative size");
    return HF_ERR_INVALID_ARG;
  }
  int64_t n = n_u + n_p;
  if (n > NA_MAX_N) {
    char buf[160];
    snprintf(buf, sizeof buf, "hf_increment_norms_noalloc: %lld unknowns exceed the fixed scratch limit of %lld",
             (long long)n, (long long)NA_MAX_N);
    set_msg(err, err_len, buf);
    return HF_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
    set_msg(err, err_len, "hf_increment_norms_noalloc: no usable current device");
    return HF_ERR_CUDA;
  }
  // the device address of the static scratch: looked up on the first call on
  // each device, and again on every call whose stream is not being captured,
  // so that an address cached before a device reset (which reloads the
  // library's device module) is never used; a call inside a stream capture
  // uses the address of the last call made outside one
  double* sc = nullptr;
  {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t qe = cudaStreamIsCapturing(st, &cs);
    if (qe != cudaSuccess) cudaGetLastError();  // the query's own error is not sticky; keep it out of later checks
    const bool capturing = qe != cudaSuccess || cs != cudaStreamCaptureStatusNone;
    std::lock_guard<std::mutex> g(na_mutex);
    if (!na_ptr[dev] || !capturing) {
      void* p = nullptr;
      cudaError_t e = capturing ? cudaErrorStreamCaptureUnsupported : cudaGetSymbolAddress(&p, na_scratch);
      if (e != cudaSuccess || !p) {
        set_msg(err, err_len,
                capturing ? "hf_increment_norms_noalloc: first call on this device made during stream capture"
                          : "hf_increment_norms_noalloc: cudaGetSymbolAddress failed");
        return HF_ERR_CUDA;
      }
      na_ptr[dev] = static_cast<double*>(p);
    }
    sc = na_ptr[dev];
  }
  if (n == 0) {
    if (cudaMemsetAsync(d_out, 0, 4 * sizeof(double), st) != cudaSuccess) return HF_ERR_CUDA;
    return HF_OK;
  }
  // the ticket must start at zero; the previous call's value is not trusted
  if (cudaMemsetAsync(sc + NA_TICKET, 0, sizeof(unsigned int), st) != cudaSuccess) {
    set_msg(err, err_len, "hf_increment_norms_noalloc: clearing the ticket failed");
    return HF_ERR_CUDA;
  }
  int blocks = (int)((n + NA_CHUNK - 1) / NA_CHUNK);
  k_increment_norms_noalloc<<<blocks, NA_THREADS, 0, st>>>(d_dx, d_x, n_u, n, d_out, sc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_msg(err, err_len, cudaGetErrorString(e));
    return HF_ERR_CUDA;
  }
  return HF_OK;
}
