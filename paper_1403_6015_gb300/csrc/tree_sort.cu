// Point ordering (Sec. 3: points sorted so that tree nodes are contiguous index ranges,
// split by point count, one dimension at a time). 1-D: one stable sort by coordinate, ties
// broken by the caller's index. 2-D: at depth t every node is sorted by coordinate t mod 2
// (ties by index) and split into its first floor(m/2) points and the rest.
//
// Stable LSD radix sort on 64-bit keys, 8-bit digits, three kernels per pass (per-chunk
// digit histogram, one-block exclusive scan in digit-major order, stable scatter with
// warp-match ranking). HBM-bound: each pass reads and writes 12 bytes per point.
#include <cuda_runtime.h>

#include "hodlr_internal.cuh"

namespace hodlr {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kChunk = kSortThreads * kSortItems;  // keys per block

// Order-preserving map from double to uint64 (after folding -0.0 into +0.0).
__device__ __forceinline__ uint64_t key_of(double v) {
  v = v + 0.0;
  uint64_t b = (uint64_t)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void k_init_coord_keys(const double* __restrict__ x, int d, int dim, int64_t n,
                                  uint64_t* __restrict__ key, int32_t* __restrict__ val) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  key[i] = key_of(x[i * d + dim]);
  val[i] = (int32_t)i;
}

__global__ void k_hist(const uint64_t* __restrict__ key, int64_t n, int shift, int nblk,
                       uint32_t* __restrict__ counts) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kChunk;
  for (int it = 0; it < kSortItems; ++it) {
    int64_t i = base + it * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(key[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  counts[(int64_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of m entries by one block of 1024 threads, in tiles of 1024 x kScanT
// entries: a tile is loaded coalesced into shared memory (padded by one word per 32 so
// that each thread's kScanT contiguous entries sit in distinct banks), every thread sums
// its entries, the 1024 sums are scanned by warp shuffles and then across the 32 warp
// totals, and the tile is written back coalesced, offset by the running carry of the
// tiles before it.
constexpr int kScanT = 8;
constexpr int kScanTile = 1024 * kScanT;

__device__ __forceinline__ int scan_pad(int j) { return j + (j >> 5); }

__global__ void __launch_bounds__(1024) k_scan(uint32_t* __restrict__ a, int64_t m) {
  __shared__ uint32_t s[kScanTile + kScanTile / 32];
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t carry_next;
  int t = threadIdx.x, lane = t & 31, w = t >> 5;
  uint32_t carry = 0;
  for (int64_t base = 0; base < m; base += kScanTile) {
#pragma unroll
    for (int q = 0; q < kScanT; ++q) {
      int j = q * 1024 + t;
      s[scan_pad(j)] = base + j < m ? a[base + j] : 0u;
    }
    __syncthreads();
    uint32_t v[kScanT], sum = 0;
#pragma unroll
    for (int q = 0; q < kScanT; ++q) {
      v[q] = s[scan_pad(t * kScanT + q)];
      sum += v[q];
    }
    uint32_t x = sum;  // inclusive scan of the thread sums within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
      uint32_t y = wsum[lane], z = y;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t u = __shfl_up_sync(0xffffffffu, z, o);
        if (lane >= o) z += u;
      }
      wsum[lane] = z - y;  // exclusive prefix of the warp totals
    }
    __syncthreads();
    uint32_t run = carry + wsum[w] + (x - sum);
#pragma unroll
    for (int q = 0; q < kScanT; ++q) {
      s[scan_pad(t * kScanT + q)] = run;
      run += v[q];
    }
    if (t == 1023) carry_next = run;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kScanT; ++q) {
      int j = q * 1024 + t;
      if (base + j < m) a[base + j] = s[scan_pad(j)];
    }
    carry = carry_next;
    __syncthreads();  // the next tile overwrites s and carry_next
  }
}

__global__ void k_scatter(const uint64_t* __restrict__ key, const int32_t* __restrict__ val,
                          int64_t n, int shift, int nblk, const uint32_t* __restrict__ offs,
                          uint64_t* __restrict__ okey, int32_t* __restrict__ oval) {
  __shared__ uint32_t base[256];
  __shared__ uint32_t run[256];
  __shared__ uint32_t wc[kSortThreads / 32][257];
  int t = threadIdx.x, lane = t & 31, w = t >> 5;
  base[t] = offs[(int64_t)t * nblk + blockIdx.x];
  run[t] = 0;
  for (int q = 0; q < kSortThreads / 32; ++q) wc[q][t] = 0;
  __syncthreads();
  int64_t b0 = (int64_t)blockIdx.x * kChunk;
  unsigned lt = (1u << lane) - 1u;
  for (int it = 0; it < kSortItems; ++it) {
    int64_t i = b0 + it * kSortThreads + t;
    bool ok = i < n;
    uint64_t k = ok ? key[i] : 0;
    int32_t v = ok ? val[i] : 0;
    unsigned dig = ok ? (unsigned)((k >> shift) & 255u) : 256u;
    unsigned peers = __match_any_sync(0xffffffffu, dig);
    unsigned rk = __popc(peers & lt);
    if (ok && lane == __ffs(peers) - 1) wc[w][dig] = __popc(peers);
    __syncthreads();
    if (ok) {
      uint32_t pos = base[dig] + run[dig] + rk;
      for (int q = 0; q < w; ++q) pos += wc[q][dig];
      okey[pos] = k;
      oval[pos] = v;
    }
    __syncthreads();
    uint32_t tot = 0;
    for (int q = 0; q < kSortThreads / 32; ++q) {
      tot += wc[q][t];
      wc[q][t] = 0;
    }
    run[t] += tot;
    __syncthreads();
  }
}

__global__ void k_gather_points(const double* __restrict__ x, int d, int64_t n,
                                const int32_t* __restrict__ perm, double* __restrict__ xs) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t p = perm[i];
  for (int c = 0; c < d; ++c) xs[c * n + i] = x[p * d + c];
}

// For the kd ordering: label every point (in caller order) with the id of the level-t node
// holding its current position, found by walking down from the root.
__global__ void k_node_labels(const int32_t* __restrict__ perm, int64_t n,
                              const int32_t* __restrict__ nodes, int t,
                              uint64_t* __restrict__ key) {
  int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pos >= n) return;
  int64_t id = 0;
  for (int l = 0; l < t; ++l) {
    int64_t rc = 2 * id + 2;
    id = pos < nodes[rc] ? 2 * id + 1 : rc;
  }
  key[perm[pos]] = (uint64_t)(id - ((1ll << t) - 1));
}

// Reorder keys (given per caller index) into the current sequence `val`.
__global__ void k_take_keys(const uint64_t* __restrict__ src, const int32_t* __restrict__ val,
                            int64_t n, uint64_t* __restrict__ dst) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[val[i]];
}

struct SortBufs {
  uint64_t *k0 = nullptr, *k1 = nullptr, *kaux = nullptr;
  int32_t *v0 = nullptr, *v1 = nullptr;
  uint32_t* counts = nullptr;
  int nblk = 0;
  cudaError_t alloc(int64_t n, bool aux) {
    nblk = (int)((n + kChunk - 1) / kChunk);
    HODLR_CUDA_TRY(cudaMalloc(&k0, n * 8));
    HODLR_CUDA_TRY(cudaMalloc(&k1, n * 8));
    if (aux) HODLR_CUDA_TRY(cudaMalloc(&kaux, n * 8));
    HODLR_CUDA_TRY(cudaMalloc(&v0, n * 4));
    HODLR_CUDA_TRY(cudaMalloc(&v1, n * 4));
    HODLR_CUDA_TRY(cudaMalloc(&counts, (size_t)256 * nblk * 4));
    return cudaSuccess;
  }
  void release() {
    cudaFree(k0); cudaFree(k1); cudaFree(kaux); cudaFree(v0); cudaFree(v1); cudaFree(counts);
  }
};

// Stable sort of (k0, v0) by key bits [0, bits); result back in (k0, v0).
cudaError_t radix_passes(SortBufs& b, int64_t n, int bits, cudaStream_t s, int64_t* launches) {
  for (int shift = 0; shift < bits; shift += 8) {
    *launches += 3;
    k_hist<<<b.nblk, kSortThreads, 0, s>>>(b.k0, n, shift, b.nblk, b.counts);
    k_scan<<<1, 1024, 0, s>>>(b.counts, (int64_t)256 * b.nblk);
    k_scatter<<<b.nblk, kSortThreads, 0, s>>>(b.k0, b.v0, n, shift, b.nblk, b.counts, b.k1, b.v1);
    std::swap(b.k0, b.k1);
    std::swap(b.v0, b.v1);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sort_1d(Ctx& c, const double* x) {
  int64_t n = c.n;
  SortBufs b;
  cudaError_t e = b.alloc(n, false);
  if (e == cudaSuccess) {
    int g = (int)((n + 255) / 256);
    k_init_coord_keys<<<g, 256, 0, c.stream>>>(x, 1, 0, n, b.k0, b.v0);
    ++c.launches;
    e = radix_passes(b, n, 64, c.stream, &c.launches);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.perm, b.v0, n * 4, cudaMemcpyDeviceToDevice, c.stream);
    k_gather_points<<<g, 256, 0, c.stream>>>(x, 1, n, c.perm, c.xs);
    ++c.launches;
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    ++c.syncs;
  }
  b.release();
  return e;
}

cudaError_t launch_sort_kd(Ctx& c, const double* x) {
  int64_t n = c.n;
  SortBufs b;
  cudaError_t e = b.alloc(n, true);
  int g = (int)((n + 255) / 256);
  int levels = c.kappa > 0 ? c.kappa : 1;
  if (e == cudaSuccess) {
    // identity order before depth 0
    k_init_coord_keys<<<g, 256, 0, c.stream>>>(x, c.d, 0, n, b.k0, b.v0);
    ++c.launches;
    e = cudaMemcpyAsync(c.perm, b.v0, n * 4, cudaMemcpyDeviceToDevice, c.stream);
  }
  for (int t = 0; t < levels && e == cudaSuccess; ++t) {
    int dim = t % c.d;
    // caller-order sequence keyed by coordinate, stably sorted: ties keep caller order
    k_init_coord_keys<<<g, 256, 0, c.stream>>>(x, c.d, dim, n, b.k0, b.v0);
    ++c.launches;
    e = radix_passes(b, n, 64, c.stream, &c.launches);
    if (e != cudaSuccess || t == 0) {
      if (e == cudaSuccess) e = cudaMemcpyAsync(c.perm, b.v0, n * 4, cudaMemcpyDeviceToDevice, c.stream);
      continue;
    }
    // labels of the level-t nodes (from the previous depth's order), then a stable sort by
    // label: the result is grouped by node, sorted by coordinate, ties by caller index
    k_node_labels<<<g, 256, 0, c.stream>>>(c.perm, n, c.nodes, t, b.kaux);
    ++c.launches;
    k_take_keys<<<g, 256, 0, c.stream>>>(b.kaux, b.v0, n, b.k0);
    ++c.launches;
    int bits = 8 * ((t + 7) / 8);
    e = radix_passes(b, n, bits, c.stream, &c.launches);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.perm, b.v0, n * 4, cudaMemcpyDeviceToDevice, c.stream);
  }
  if (e == cudaSuccess) {
    k_gather_points<<<g, 256, 0, c.stream>>>(x, c.d, n, c.perm, c.xs);
    ++c.launches;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  ++c.syncs;
  b.release();
  return e;
}

}  // namespace hodlr
