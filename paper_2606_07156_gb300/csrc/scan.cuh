// ADC inner loops shared by the search kernels (DC of Section 2.1).
//
// A lane holds one vector's packed codes (NCHUNK 16-byte chunks, byte m is the
// code of sub-space m) and sums its LUT entries T[m][code_m] over m < Mp.
// Tables live in shared memory, row m at element offset m*256. Every lookup
// is one 32-bit shared load at [address + m*256*sizeof(entry)], the row
// offset being an immediate: the sub-space index is a template parameter,
// expanded by a fold over m.
#pragma once

#include <stdint.h>

#include <utility>

#include "common.cuh"

namespace anns {

template <int OFF>
__device__ __forceinline__ uint32_t lds_u8(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u8 %0, [%1+%2];" : "=r"(v) : "r"(a), "n"(OFF));
  return v;
}
template <int OFF>
__device__ __forceinline__ uint32_t lds_u16(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u16 %0, [%1+%2];" : "=r"(v) : "r"(a), "n"(OFF));
  return v;
}
template <int OFF>
__device__ __forceinline__ float lds_f32(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(a), "n"(OFF));
  return v;
}

// Packed code word holding sub-spaces K..K+3 (K a multiple of 4).
template <int K, int NCHUNK>
__device__ __forceinline__ uint32_t code_word(const uint4 (&w)[NCHUNK]) {
  constexpr int c = K / 16, i = (K % 16) / 4;
  if constexpr (i == 0) return w[c].x;
  else if constexpr (i == 1) return w[c].y;
  else if constexpr (i == 2) return w[c].z;
  else return w[c].w;
}

// Table entry of sub-space K for the vector whose codes are w. `base` is the
// table's shared-memory byte address; for uint8 tables it must have a zero
// low byte (the code is merged in by one byte-permute).
template <typename LT, int K, int NCHUNK>
__device__ __forceinline__ auto lut_entry(uint32_t base, const uint4 (&w)[NCHUNK]) {
  const uint32_t x = code_word<K & ~3, NCHUNK>(w);
  if constexpr (sizeof(LT) == 1) {
    return lds_u8<K * 256>(__byte_perm(x, base, 0x7650u + (K & 3)));
  } else {
    const uint32_t code = __byte_perm(x, 0u, 0x4440u + (K & 3));
    if constexpr (sizeof(LT) == 2) return lds_u16<K * 512>(base + code * 2u);
    else return lds_f32<K * 1024>(base + code * 4u);
  }
}

// S = sum_m t[m][code_m] over m < Mp, exact (integer tables).
template <typename LT, int NCHUNK, int... K>
__device__ __forceinline__ int adc_int_seq(uint32_t base, const uint4 (&w)[NCHUNK],
                                           std::integer_sequence<int, K...>) {
  return (0 + ... + (int)lut_entry<LT, K, NCHUNK>(base, w));
}
template <typename LT, int NCHUNK>
__device__ __forceinline__ int adc_int(uint32_t base, const uint4 (&w)[NCHUNK]) {
  return adc_int_seq<LT, NCHUNK>(base, w, std::make_integer_sequence<int, NCHUNK * 16>{});
}

// acc = fl32(acc + T[m][code_m]) for m = 0..Mp-1 ascending (FP32 tables).
template <int NCHUNK, int... K>
__device__ __forceinline__ float adc_f32_seq(uint32_t base, const uint4 (&w)[NCHUNK],
                                             std::integer_sequence<int, K...>) {
  float acc = 0.f;
  ((acc = add_rn(acc, lut_entry<float, K, NCHUNK>(base, w))), ...);
  return acc;
}
template <int NCHUNK>
__device__ __forceinline__ float adc_f32(uint32_t base, const uint4 (&w)[NCHUNK]) {
  return adc_f32_seq<NCHUNK>(base, w, std::make_integer_sequence<int, NCHUNK * 16>{});
}

// Shared-memory byte address of a generic pointer into this block's shared memory.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

}  // namespace anns
