// lb_series.cu -- analysis of a shear-response record on the device: the
// bursts of the response's time derivative and the waiting times between
// them (Sec. VIII, Fig. 14: intermittent bursts of dU/dt whose spacing is
// power-law distributed).
//
// The record holds U_k after every step in a ring (lb_kernels.h, Series).
// With d_j = U_{j+1} - U_j over the held entries, mu and sigma the mean and
// population standard deviation of d, step j is "above" when
// |d_j - mu| > c sigma; a burst is a maximal run of above steps starting at
// its first step; waits are the differences of successive burst starts,
// counted in bins [2^b, 2^(b+1)).  One CTA walks the record in chunks: a
// reduction for mu and sigma, then per chunk a ballot/scan compaction of the
// burst starts (in order) and the waits to their predecessors.
#include <math.h>

#include "lb_kernels.h"

namespace lbk {

constexpr int SB = 1024;        // threads of the analysis CTA
constexpr int kMaxBurstBins = 64;

__device__ __forceinline__ double rec_entry(const Series& sr, long long base, long long j,
                                            double scale) {
  return scale * sr.buf[(base + j) % sr.cap];
}

__global__ void __launch_bounds__(SB) k_series_bursts(Series sr, double scale, double c, int nbins,
                                                      long long* out) {
  __shared__ double s_a[SB / 32], s_b[SB / 32];
  __shared__ double s_mu, s_th;
  __shared__ int s_wcnt[SB / 32], s_woff[SB / 32], s_cnt;
  __shared__ int s_pos[SB];
  __shared__ long long s_last, s_events;
  __shared__ unsigned long long s_hist[kMaxBurstBins];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long t = *(volatile long long*)sr.t;
  const long long n = t < sr.cap - 1 ? t : sr.cap - 1;  // entries held
  const long long m = n - 1;                             // derivative samples
  const long long base = t - n;
  if (threadIdx.x < kMaxBurstBins) s_hist[threadIdx.x] = 0ull;
  if (threadIdx.x == 0) {
    s_last = -1;
    s_events = 0;
  }
  if (m >= 2) {
    // mean and mean square of d
    double a = 0.0, b = 0.0;
    for (long long j = threadIdx.x; j < m; j += SB) {
      const double d = rec_entry(sr, base, j + 1, scale) - rec_entry(sr, base, j, scale);
      a += d;
      b += d * d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      s_a[warp] = a;
      s_b[warp] = b;
    }
    __syncthreads();
    if (warp == 0) {
      a = s_a[lane];
      b = s_b[lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
      }
      if (lane == 0) {
        const double mu = a / (double)m;
        const double var = b / (double)m - mu * mu;
        s_mu = mu;
        s_th = c * sqrt(var > 0.0 ? var : 0.0);
      }
    }
    __syncthreads();
    const double mu = s_mu, th = s_th;
    for (long long c0 = 0; c0 < m; c0 += SB) {
      const long long j = c0 + threadIdx.x;
      bool start = false;
      if (j < m) {
        const double e1 = rec_entry(sr, base, j, scale);
        const bool above = fabs(rec_entry(sr, base, j + 1, scale) - e1 - mu) > th;
        const bool prev = j > 0 && fabs(e1 - rec_entry(sr, base, j - 1, scale) - mu) > th;
        start = above && !prev;
      }
      // ordered compaction of the chunk's burst starts
      const unsigned bal = __ballot_sync(0xffffffffu, start);
      if (lane == 0) s_wcnt[warp] = __popc(bal);
      __syncthreads();
      if (warp == 0) {
        const int v = s_wcnt[lane];
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int u = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += u;
        }
        s_woff[lane] = incl - v;
        if (lane == 31) s_cnt = incl;
      }
      __syncthreads();
      if (start) s_pos[s_woff[warp] + __popc(bal & ((1u << lane) - 1u))] = threadIdx.x;
      __syncthreads();
      const int cnt = s_cnt;
      for (int k = threadIdx.x; k < cnt; k += SB) {
        const long long pj = c0 + s_pos[k];
        const long long pp = (k == 0) ? s_last : c0 + s_pos[k - 1];
        if (pp >= 0) {
          int bin = 63 - __clzll((long long)(pj - pp));
          if (bin > nbins - 1) bin = nbins - 1;
          atomicAdd(&s_hist[bin], 1ull);
        }
      }
      __syncthreads();
      if (threadIdx.x == 0 && cnt > 0) {
        s_last = c0 + s_pos[cnt - 1];
        s_events += cnt;
      }
      __syncthreads();
    }
  }
  __syncthreads();
  if (threadIdx.x < nbins) out[2 + threadIdx.x] = (long long)s_hist[threadIdx.x];
  if (threadIdx.x == 0) {
    out[0] = s_events;
    out[1] = m > 0 ? m : 0;
  }
}

int series_bursts(const Series& sr, double scale, double c, int nbins, int64_t* hist,
                  int64_t* events, cudaStream_t st) {
  if (!sr.buf || !(c >= 0.0) || nbins < 1 || nbins > kMaxBurstBins || !hist) return LB_EINVAL;
  long long* d_out = nullptr;
  const size_t bytes = (size_t)(nbins + 2) * sizeof(long long);
  if (cudaMalloc(&d_out, bytes) != cudaSuccess) {
    cudaGetLastError();
    return LB_ENOMEM;
  }
  long long h_out[kMaxBurstBins + 2];
  k_series_bursts<<<1, SB, 0, st>>>(sr, scale, c, nbins, d_out);
  const bool ok = cudaGetLastError() == cudaSuccess &&
                  cudaMemcpyAsync(h_out, d_out, bytes, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                  cudaStreamSynchronize(st) == cudaSuccess;
  cudaFree(d_out);
  if (!ok) return LB_ECUDA;
  for (int b = 0; b < nbins; ++b) hist[b] = h_out[2 + b];
  if (events) *events = h_out[0];
  return LB_OK;
}

}  // namespace lbk
