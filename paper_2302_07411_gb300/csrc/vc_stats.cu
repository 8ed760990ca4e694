// vc_stats.cu -- the statistical and security measures of Sec. 4 and Sec. 5
// as device kernels, so the checks run on frames where they already are.
//
// Integer work (histograms, moment sums of adjacent pixels, NPCR counts,
// UACI sums) is exact; the measures are then formed in binary64 from the
// exact integers.  Random choices of the measures (which adjacent pairs,
// which blocks) are inputs.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "vcrypt.h"

namespace {

constexpr int kStatThreads = 256;

// a * b - c * d for unsigned 64-bit operands, exactly, as a double (rounded once
// per 64-bit half).
__device__ double mul_sub_mul(unsigned long long a, unsigned long long b, unsigned long long c, unsigned long long d) {
  const unsigned long long h1 = __umul64hi(a, b), l1 = a * b;
  const unsigned long long h2 = __umul64hi(c, d), l2 = c * d;
  const bool neg = h1 < h2 || (h1 == h2 && l1 < l2);
  unsigned long long hi, lo;
  if (!neg) {
    lo = l1 - l2;
    hi = h1 - h2 - (l1 < l2 ? 1 : 0);
  } else {
    lo = l2 - l1;
    hi = h2 - h1 - (l2 < l1 ? 1 : 0);
  }
  const double v = (double)hi * 18446744073709551616.0 + (double)lo;
  return neg ? -v : v;
}
constexpr int kBytesPerCta = 64 * 1024;  // bytes of one frame per histogram CTA

bool frame_ok(int nframes, int H, int W, int C) {
  return nframes >= 0 && H >= 1 && W >= 1 && (C == 1 || C == 3 || C == 4) &&
         (long long)H * W * C < (1LL << 31);
}

// Counts z[f][c][v] (Sec. 4.1).  Grid (ceil(N / kBytesPerCta), nframes); each
// CTA bins its slice in shared memory, then adds to the frame's counts.
__global__ void __launch_bounds__(kStatThreads) k_hist(const uint8_t* frames, long long N, int C,
                                                         unsigned int* hist) {
  __shared__ unsigned int s[4 * 256];
  for (int k = threadIdx.x; k < C * 256; k += blockDim.x) s[k] = 0;
  __syncthreads();
  const uint8_t* fr = frames + (long long)blockIdx.y * N;
  const long long b0 = (long long)blockIdx.x * kBytesPerCta;
  long long b1 = b0 + kBytesPerCta;
  if (b1 > N) b1 = N;
  const bool vec = ((reinterpret_cast<uintptr_t>(fr) & 15) == 0);
  if (vec) {
    const long long v0 = (b0 + 15) / 16, v1 = b1 / 16;
    for (long long v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
      const uint4 w = __ldg(reinterpret_cast<const uint4*>(fr) + v);
      const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
      int ch = (int)((v * 16) % C);
#pragma unroll
      for (int k = 0; k < 16; k++) {
        atomicAdd(&s[ch * 256 + ((ws[k >> 2] >> (8 * (k & 3))) & 0xFF)], 1u);
        if (++ch == C) ch = 0;
      }
    }
    // bytes outside whole 16-byte words
    for (long long q = b0 + threadIdx.x; q < b1; q += blockDim.x)
      if (q < v0 * 16 || q >= v1 * 16) atomicAdd(&s[(int)(q % C) * 256 + fr[q]], 1u);
  } else {
    for (long long q = b0 + threadIdx.x; q < b1; q += blockDim.x) atomicAdd(&s[(int)(q % C) * 256 + fr[q]], 1u);
  }
  __syncthreads();
  unsigned int* h = hist + (long long)blockIdx.y * C * 256;
  for (int k = threadIdx.x; k < C * 256; k += blockDim.x)
    if (s[k]) atomicAdd(&h[k], s[k]);
}

// From the counts of one (frame, channel) (one CTA of 256 threads):
// chi^2 = sum (z - e)^2 / e with e = N/256, var(Z) = (256 sum z^2 - (sum z)^2) / 256^2
// (the double sum of Sec. 4.1 in closed form, exact in integers), and the
// Shannon entropy sum p log2(1/p) (Sec. 4.3).
__global__ void __launch_bounds__(256) k_hist_measures(const unsigned int* hist, double* chi2, double* var,
                                                         double* ent) {
  __shared__ double s_a[256], s_b[256];
  __shared__ unsigned long long s_n[256], s_q[256];
  const unsigned int* h = hist + (long long)blockIdx.x * 256;
  const unsigned int z = h[threadIdx.x];
  s_n[threadIdx.x] = z;
  s_q[threadIdx.x] = (unsigned long long)z * z;
  __syncthreads();
  for (int d = 128; d > 0; d >>= 1) {
    if (threadIdx.x < d) {
      s_n[threadIdx.x] += s_n[threadIdx.x + d];
      s_q[threadIdx.x] += s_q[threadIdx.x + d];
    }
    __syncthreads();
  }
  const unsigned long long n = s_n[0], sq = s_q[0];
  const double e = (double)n / 256.0;
  const double dz = (double)z - e;
  s_a[threadIdx.x] = n ? dz * dz / e : 0.0;
  const double p = n ? (double)z / (double)n : 0.0;
  s_b[threadIdx.x] = z ? -p * log2(p) : 0.0;
  __syncthreads();
  for (int d = 128; d > 0; d >>= 1) {
    if (threadIdx.x < d) {
      s_a[threadIdx.x] += s_a[threadIdx.x + d];
      s_b[threadIdx.x] += s_b[threadIdx.x + d];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (chi2) chi2[blockIdx.x] = s_a[0];
    if (ent) ent[blockIdx.x] = s_b[0];
    if (var) var[blockIdx.x] = mul_sub_mul(256ULL, sq, n, n) / 65536.0;
  }
}

// Exact moment sums of adjacent pixel pairs (Sec. 4.2) of one frame: pair k is
// pixel p = pairs[k] (all pairs when pairs == null, k enumerating them) and its
// right (dir 0), lower (dir 1) or lower-right (dir 2) neighbour, per channel.
// sums[f][c][6] = sum x, sum y, sum x^2, sum y^2, sum x y, pairs (a given
// index whose pair leaves the frame is skipped).
__global__ void __launch_bounds__(kStatThreads) k_corr_sums(const uint8_t* frames, long long N, int H, int W, int C,
                                                              int dir, const int* pairs, long long npairs,
                                                              unsigned long long* sums) {
  const uint8_t* fr = frames + (long long)blockIdx.y * N;
  const int dy = dir == 0 ? 0 : 1, dx = dir == 1 ? 0 : 1;
  const int Wv = W - dx;  // valid first-pixel columns
  unsigned long long acc[4][5];
  unsigned long long used = 0;
#pragma unroll
  for (int c = 0; c < 4; c++)
#pragma unroll
    for (int m = 0; m < 5; m++) acc[c][m] = 0;
  auto pair = [&](long long p) {
    used++;
    const long long p2 = p + (long long)dy * W + dx;
#pragma unroll
    for (int c = 0; c < 4; c++) {
      if (c < C) {
        const unsigned int x = fr[p * C + c], y = fr[p2 * C + c];
        acc[c][0] += x;
        acc[c][1] += y;
        acc[c][2] += x * x;
        acc[c][3] += y * y;
        acc[c][4] += x * y;
      }
    }
  };
  if (pairs) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < npairs;
         k += (long long)gridDim.x * blockDim.x) {
      const long long p = pairs[k];
      if (p < 0 || p / W >= H - dy || p % W >= Wv) continue;
      pair(p);
    }
  } else {
    // every pair: CTAs take rows, threads take consecutive columns
    for (int row = blockIdx.x; row < H - dy; row += gridDim.x)
      for (int col = threadIdx.x; col < Wv; col += blockDim.x) pair((long long)row * W + col);
  }
  // warp reduction, then one atomic per warp and quantity
#pragma unroll
  for (int c = 0; c < 4; c++) {
    if (c >= C) break;
#pragma unroll
    for (int m = 0; m < 6; m++) {
      unsigned long long v = m < 5 ? acc[c][m] : used;
      for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, d);
      if ((threadIdx.x & 31) == 0 && v) atomicAdd(&sums[((long long)blockIdx.y * C + c) * 6 + m], v);
    }
  }
}

// r = cov(x, y) / sqrt(D(x) D(y)) with 1/N moments, from the exact sums:
// (N sxy - sx sy) / sqrt((N sxx - sx^2)(N syy - sy^2)).
__global__ void k_corr_finish(const unsigned long long* sums, int count, double* r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const unsigned long long* s = sums + (long long)i * 6;
  const unsigned long long n = s[5];
  const double num = mul_sub_mul(n, s[4], s[0], s[1]);
  const double dxx = mul_sub_mul(n, s[2], s[0], s[0]);
  const double dyy = mul_sub_mul(n, s[3], s[1], s[1]);
  r[i] = num / sqrt(dxx * dyy);
}

// Local entropy (Sec. 4.3): entropy of block b (side x side pixels of channel
// ch, top-left (blocks[2b], blocks[2b+1])) of frame f; one CTA per (b, f).
__global__ void __launch_bounds__(256) k_block_entropy(const uint8_t* frames, long long N, int H, int W, int C,
                                                         int ch, const int* blocks, int side, double* ent) {
  __shared__ unsigned int s[256];
  __shared__ double sh[256];
  s[threadIdx.x] = 0;
  __syncthreads();
  const uint8_t* fr = frames + (long long)blockIdx.y * N;
  const int y0 = blocks[2 * blockIdx.x], x0 = blocks[2 * blockIdx.x + 1];
  if (y0 < 0 || x0 < 0 || y0 > H - side || x0 > W - side) {  // a block outside the frame
    if (threadIdx.x == 0) ent[(long long)blockIdx.y * gridDim.x + blockIdx.x] = nan("");
    return;
  }
  const int tot = side * side;
  for (int k = threadIdx.x; k < tot; k += blockDim.x) {
    const int yy = k / side, xx = k - yy * side;
    atomicAdd(&s[fr[((long long)(y0 + yy) * W + (x0 + xx)) * C + ch]], 1u);
  }
  __syncthreads();
  const double p = (double)s[threadIdx.x] / (double)tot;
  sh[threadIdx.x] = s[threadIdx.x] ? -p * log2(p) : 0.0;
  __syncthreads();
  for (int d = 128; d > 0; d >>= 1) {
    if (threadIdx.x < d) sh[threadIdx.x] += sh[threadIdx.x + d];
    __syncthreads();
  }
  if (threadIdx.x == 0) ent[(long long)blockIdx.y * gridDim.x + blockIdx.x] = sh[0];
}

// Mean of the k block entropies of each frame (in block order, as summed on the host side).
__global__ void k_block_mean(const double* ent, int k, int nframes, double* out) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nframes) return;
  double s = 0.0;
  for (int b = 0; b < k; b++) s += ent[(long long)f * k + b];
  out[f] = s / k;
}

// NPCR / UACI counts (Sec. 5.2) of frame pair f: per channel, the number of
// differing bytes and the sum of |a - b|.
__global__ void __launch_bounds__(kStatThreads) k_npcr_sums(const uint8_t* a, const uint8_t* b, long long N, int C,
                                                              unsigned long long* sums) {
  const uint8_t* fa = a + (long long)blockIdx.y * N;
  const uint8_t* fb = b + (long long)blockIdx.y * N;
  unsigned long long cnt[4] = {0, 0, 0, 0}, sad[4] = {0, 0, 0, 0};
  auto add = [&](int c, unsigned int x, unsigned int y) {
    const unsigned int ad = x > y ? x - y : y - x;
#pragma unroll
    for (int k = 0; k < 4; k++)
      if (k == c) {
        cnt[k] += ad != 0;
        sad[k] += ad;
      }
  };
  const long long stride = (long long)gridDim.x * blockDim.x;
  if (((reinterpret_cast<uintptr_t>(fa) | reinterpret_cast<uintptr_t>(fb)) & 15) == 0) {
    // 16 bytes per step, the channel of byte k rotating from (16 v) mod C
    const long long nv = N / 16;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) {
      const uint4 wa = __ldg(reinterpret_cast<const uint4*>(fa) + v);
      const uint4 wb = __ldg(reinterpret_cast<const uint4*>(fb) + v);
      const uint32_t xa[4] = {wa.x, wa.y, wa.z, wa.w}, xb[4] = {wb.x, wb.y, wb.z, wb.w};
      int c = (int)((v * 16) % C);
#pragma unroll
      for (int k = 0; k < 16; k++) {
        add(c, (xa[k >> 2] >> (8 * (k & 3))) & 0xFFu, (xb[k >> 2] >> (8 * (k & 3))) & 0xFFu);
        if (++c == C) c = 0;
      }
    }
    for (long long q = nv * 16 + (long long)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += stride)
      add((int)(q % C), fa[q], fb[q]);
  } else {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += stride)
      add((int)(q % C), fa[q], fb[q]);
  }
#pragma unroll
  for (int c = 0; c < 4; c++) {
    if (c >= C) break;
    unsigned long long v0 = cnt[c], v1 = sad[c];
    for (int d = 16; d > 0; d >>= 1) {
      v0 += __shfl_down_sync(0xFFFFFFFFu, v0, d);
      v1 += __shfl_down_sync(0xFFFFFFFFu, v1, d);
    }
    if ((threadIdx.x & 31) == 0) {
      if (v0) atomicAdd(&sums[((long long)blockIdx.y * C + c) * 2], v0);
      if (v1) atomicAdd(&sums[((long long)blockIdx.y * C + c) * 2 + 1], v1);
    }
  }
}

__global__ void k_npcr_finish(const unsigned long long* sums, long long P, int count, double* npcr, double* uaci) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  npcr[i] = (double)sums[2 * i] / (double)P * 100.0;
  uaci[i] = (double)sums[2 * i + 1] / (double)P / 255.0 * 100.0;
}

int grid_for(long long work, int per_block_items) {
  long long g = (work + per_block_items - 1) / per_block_items;
  if (g < 1) g = 1;
  if (g > 4096) g = 4096;
  return (int)g;
}

}  // namespace

extern "C" {

int vc_stats_histogram(const uint8_t* d_frames, int32_t nframes, int32_t height, int32_t width, int32_t channels,
                       uint32_t* d_hist, double* d_chi2, double* d_var, double* d_entropy, void* stream) {
  if (!frame_ok(nframes, height, width, channels) || (nframes > 0 && (!d_frames || !d_hist))) return VC_ERR_ARG;
  if (nframes == 0) return VC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const long long N = (long long)height * width * channels;
  if (cudaMemsetAsync(d_hist, 0, sizeof(uint32_t) * 256 * channels * (size_t)nframes, st) != cudaSuccess)
    return VC_ERR_CUDA;
  dim3 grid((unsigned)((N + kBytesPerCta - 1) / kBytesPerCta), (unsigned)nframes);
  k_hist<<<grid, kStatThreads, 0, st>>>(d_frames, N, channels, d_hist);
  if (d_chi2 || d_var || d_entropy)
    k_hist_measures<<<nframes * channels, 256, 0, st>>>(d_hist, d_chi2, d_var, d_entropy);
  return cudaGetLastError() == cudaSuccess ? VC_OK : VC_ERR_CUDA;
}

int vc_stats_correlation(const uint8_t* d_frames, int32_t nframes, int32_t height, int32_t width, int32_t channels,
                         int32_t direction, const int32_t* d_pairs, int64_t npairs, uint64_t* d_sums, double* d_r,
                         void* stream) {
  if (!frame_ok(nframes, height, width, channels) || direction < 0 || direction > 2 || !d_sums || !d_r)
    return VC_ERR_ARG;
  const int dy = direction == 0 ? 0 : 1, dx = direction == 1 ? 0 : 1;
  const long long all = (long long)(height - dy) * (width - dx);
  if (!d_pairs) npairs = all;
  if (npairs < 2 || (d_pairs && npairs > (1LL << 31))) return VC_ERR_ARG;
  if (nframes == 0) return VC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const long long N = (long long)height * width * channels;
  const int count = nframes * channels;
  if (cudaMemsetAsync(d_sums, 0, sizeof(uint64_t) * 6 * (size_t)count, st) != cudaSuccess) return VC_ERR_CUDA;
  // all pairs: 32 CTAs per frame striding over its rows (each CTA's warps end
  // with one atomic per sum: few enough not to queue on the frame's counters)
  dim3 grid((unsigned)(d_pairs ? grid_for(npairs, kStatThreads * 16) : (height - dy < 32 ? height - dy : 32)),
            (unsigned)nframes);
  k_corr_sums<<<grid, kStatThreads, 0, st>>>(d_frames, N, height, width, channels, direction,
                                             reinterpret_cast<const int*>(d_pairs), npairs,
                                             reinterpret_cast<unsigned long long*>(d_sums));
  k_corr_finish<<<(count + 127) / 128, 128, 0, st>>>(reinterpret_cast<const unsigned long long*>(d_sums), count, d_r);
  return cudaGetLastError() == cudaSuccess ? VC_OK : VC_ERR_CUDA;
}

int vc_stats_local_entropy(const uint8_t* d_frames, int32_t nframes, int32_t height, int32_t width, int32_t channels,
                           int32_t channel, const int32_t* d_blocks, int32_t nblocks, int32_t side, double* d_block_ent,
                           double* d_mean, void* stream) {
  if (!frame_ok(nframes, height, width, channels) || channel < 0 || channel >= channels || nblocks < 1 ||
      nblocks > 65535 || side < 1 || side > height || side > width || !d_blocks || !d_block_ent || !d_mean)
    return VC_ERR_ARG;
  if (nframes == 0) return VC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const long long N = (long long)height * width * channels;
  dim3 grid((unsigned)nblocks, (unsigned)nframes);
  k_block_entropy<<<grid, 256, 0, st>>>(d_frames, N, height, width, channels, channel,
                                        reinterpret_cast<const int*>(d_blocks), side, d_block_ent);
  k_block_mean<<<(nframes + 127) / 128, 128, 0, st>>>(d_block_ent, nblocks, nframes, d_mean);
  return cudaGetLastError() == cudaSuccess ? VC_OK : VC_ERR_CUDA;
}

int vc_stats_npcr_uaci(const uint8_t* d_a, const uint8_t* d_b, int32_t nframes, int32_t height, int32_t width,
                       int32_t channels, uint64_t* d_sums, double* d_npcr, double* d_uaci, void* stream) {
  if (!frame_ok(nframes, height, width, channels) || (nframes > 0 && (!d_a || !d_b)) || !d_sums || !d_npcr ||
      !d_uaci)
    return VC_ERR_ARG;
  if (nframes == 0) return VC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const long long N = (long long)height * width * channels;
  const int count = nframes * channels;
  if (cudaMemsetAsync(d_sums, 0, sizeof(uint64_t) * 2 * (size_t)count, st) != cudaSuccess) return VC_ERR_CUDA;
  dim3 grid((unsigned)grid_for(N, kStatThreads * 16), (unsigned)nframes);
  k_npcr_sums<<<grid, kStatThreads, 0, st>>>(d_a, d_b, N, channels, reinterpret_cast<unsigned long long*>(d_sums));
  k_npcr_finish<<<(count + 127) / 128, 128, 0, st>>>(reinterpret_cast<const unsigned long long*>(d_sums),
                                                     (long long)height * width, count, d_npcr, d_uaci);
  return cudaGetLastError() == cudaSuccess ? VC_OK : VC_ERR_CUDA;
}

}  // extern "C"
