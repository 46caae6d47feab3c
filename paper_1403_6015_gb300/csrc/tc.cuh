// Fifth-generation tensor cores (tcgen05) for the double-float leaf stage: inline PTX for
// tensor-memory allocation, the shared-memory operand descriptors, the bf16 MMA with FP32
// accumulation in tensor memory, its completion through an mbarrier, and the loads of the
// accumulators back to registers. Written for sm_103a, one CTA per MMA (cta_group::1).
//
// Exact double-float products on bf16 tensor cores (after Ozaki's error-free splitting,
// "Error-free transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 2012, here with bf16 slices):
// every row of the left operand (and every column of the right one) is scaled by a power
// of two 2^e that bounds its entries, and each scaled entry v in (-1, 1) is cut into
// kSlices slices v = sum_s q_s 2^(-8(s+1)), q_0 in [-256, 256] and q_s in [-256, 256] for
// s > 0 (round to nearest at each cut), stored at their true scale. A slice has at most
// eight significant bits, so it is exact in bf16, and so is every product of two slices
// (at most 16 bits). The products of one level L = s + t all lie on the grid 2^(-8(L+2))
// and a K = 32 sum of them (at most L + 1 pairs) stays below 2^23 grid units: the FP32
// accumulation of the tensor core adds them exactly. Levels 0..4 get an accumulator each;
// levels 5..kSlices-1 share the last one, where the FP32 rounding is below 2^-56 of the
// row and column bounds (the products being summed are below 2^-40 of them). The
// accumulators are summed in double-float:
//   sum_k a_ik b_kj = 2^(e_i + f_j) (D_0 + D_1 + ... + D_5)[i][j].
// With kSlices = 7 the slicing remainder is below 2^-57 of the bound and the dropped
// levels (L >= 7) below 2^-63 per term: the result carries double-float accuracy.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "ff.cuh"

namespace hodlr {
namespace tc {

constexpr int kSlices = 7;   // bf16 slices per double-float operand
constexpr int kAcc = 6;      // accumulators: levels 0, 1, 2, 3, 4 and 5..kSlices-1 together

// Accumulator of level L = s + t.
__host__ __device__ constexpr int acc_of(int L) { return L < kAcc - 1 ? L : kAcc - 1; }

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- tensor memory ---------------------------------------------------------------------
// Allocate ncols columns (a power of two, >= 32) of tensor memory; executed by one whole
// warp; the base address is written to *slot (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                   smem_addr(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
// Generic-proxy writes to shared memory made visible to the tensor core (async proxy).
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// ---- mbarrier --------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

// Wait for the phase with the given parity to complete; gives up after max_iter polls and
// returns false (the caller records the timeout; no thread waits forever). Each poll may
// suspend the thread for up to kSuspendNs (it resumes as soon as the phase completes), so
// waiting warps leave the issue slots to the co-resident CTA; max_iter polls bound the
// wait to max_iter * kSuspendNs.
constexpr uint32_t kSuspendNs = 20000;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int max_iter) {
  uint32_t a = smem_addr(bar);
  for (int it = 0; it < max_iter; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity), "r"(kSuspendNs)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Arrive on the mbarrier once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_addr(bar))
      : "memory");
}

// ---- descriptors -----------------------------------------------------------------------
// Shared-memory operand descriptor, no swizzle, K-major: the operand is a grid of core
// matrices of 8 rows x 16 bytes (8 bf16 along K), each stored as 128 contiguous bytes
// (row-major); core matrices adjacent along K lie lbo bytes apart, adjacent along M (or N)
// sbo bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of sm_100-class tensor cores
  // base offset 0, absolute LBO mode off, layout type 0 (no swizzle)
  return d;
}

// Instruction descriptor of kind::f16 with bf16 A and B, FP32 accumulator, both operands
// K-major, dense, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4)                       // D format: F32
         | (1u << 7)                     // A format: BF16
         | (1u << 10)                    // B format: BF16
         | ((uint32_t)(N >> 3) << 17)    // N / 8
         | ((uint32_t)(M >> 4) << 24);   // M / 16
}

// D[tmem] (+)= A[smem] * B[smem]^T, one K = 16 step; issued by a single thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, bool accumulate) {
  uint32_t acc = accumulate ? 1u : 0u;
  asm volatile(
      "{\n .reg .pred p;\n"
      " setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

// ---- accumulator loads -----------------------------------------------------------------
// Eight consecutive 32-bit columns of this thread's tensor-memory lane (warp w reads lanes
// 32 (w % 4) .. 32 (w % 4) + 31; taddr carries the lane base in bits 31..16). The wait for
// the load sits in the same asm statement, so no use of the values can be scheduled
// before the data has arrived.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Four consecutive columns (as tmem_ld8).
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float* v) {
  uint32_t r[4];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- operand layout --------------------------------------------------------------------
// One slice of an operand tile of R rows (a multiple of 8) and K = 32 columns, as bf16 core
// matrices: element (r, k) at byte ((k / 8) * R / 8 + r / 8) * 128 + (r % 8) * 16 + (k % 8) * 2.
// Along K the core matrices are R * 16 bytes apart (lbo), along the rows 128 (sbo). A K = 16
// MMA step h starts 2 h core matrices further along K.
__host__ __device__ constexpr uint32_t slice_bytes(int R) { return (uint32_t)R * 32 * 2; }
__device__ __forceinline__ uint32_t slice_off(int R, int r, int k) {
  return (uint32_t)((((k >> 3) * (R >> 3) + (r >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// Exponent e with |v| < 2^e for every |v| <= m (e = 0 for m = 0).
__device__ __forceinline__ int bound_exp(float m) {
  int e = 0;
  if (m > 0.0f) frexpf(m, &e);
  return e;
}

// v * 2^e, exact for both words (barring underflow of the low word).
__device__ __forceinline__ ff ff_ldexp(ff v, int e) {
  if (e >= -126 && e <= 127) {
    float s = __int_as_float((e + 127) << 23);
    return ff{v.hi * s, v.lo * s};
  }
  return ff{ldexpf(v.hi, e), ldexpf(v.lo, e)};
}

// Cut eight double-floats v = h + l (|v| < 1 after scaling) into kSlices slices each;
// slice s of the eight values is packed as eight bf16 (one 16-byte core-matrix row) into
// out[s]. Rounding to the grid g = 2^(-8(s+1)) is (r + C) - C with C = 1.5 2^23 g, and the
// remainder r - slice is exact. Slices 0..2 come from h (24 bits); the exact remainder of
// h and l are then renormalised by a two-sum, slices 3..5 come from the new high word and
// slice 6 from what is left of it plus the low word. 28 FP32 additions per value.
__device__ __forceinline__ void cut8(const ff* v, uint4* out) {
  static_assert(kSlices == 7, "cut8 is written for seven slices");
  float h[8], l[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    h[k] = v[k].hi;
    l[k] = v[k].lo;
  }
#pragma unroll
  for (int s = 0; s < kSlices; ++s) {
    const float C = 1.5f * __int_as_float((127 + 23 - 8 * (s + 1)) << 23);
    if (s == 3) {
#pragma unroll
      for (int k = 0; k < 8; ++k) two_sum(h[k], l[k], h[k], l[k]);
    }
    if (s == 6) {
#pragma unroll
      for (int k = 0; k < 8; ++k) h[k] += l[k];
    }
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
      float q0 = (h[k] + C) - C;
      float q1 = (h[k + 1] + C) - C;
      h[k] -= q0;
      h[k + 1] -= q1;
      __nv_bfloat162 pr = __floats2bfloat162_rn(q0, q1);  // <= 8 significant bits: exact
      w[k >> 1] = *reinterpret_cast<uint32_t*>(&pr);
    }
    out[s] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// x - 2^e (D_0 + ... + D_5) in one compensated sum: both words of x and every scaled
// accumulator (exact: a power-of-two scaling) enter by error-free two-sums, whose errors
// are collected and added once. The result carries only the rounding of its own
// magnitude, also where x and the product sum nearly cancel.
__device__ __forceinline__ ff sub_acc(ff x, const float* d, int e) {
  float sc = (e >= -126 && e <= 127) ? __int_as_float((e + 127) << 23) : 0.0f;
  float s = x.hi, err = x.lo;
#pragma unroll
  for (int a = 0; a < kAcc; ++a) {
    float v = sc != 0.0f ? -d[a] * sc : -ldexpf(d[a], e);
    float t;
    two_sum(s, v, s, t);
    err += t;
  }
  ff r;
  fast_two_sum(s, err, r.hi, r.lo);
  return r;
}

// D_0 + ... + D_5 as a double-float: D_0..D_4 are exact, the terms are summed from the
// smallest by error-free two-sums with the errors collected and added once.
__device__ __forceinline__ ff combine_acc(const float* d) {
  float s = d[kAcc - 1], e = 0.0f;
#pragma unroll
  for (int a = kAcc - 2; a >= 0; --a) {
    float t;
    two_sum(d[a], s, s, t);
    e += t;
  }
  ff r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

}  // namespace tc
}  // namespace hodlr
