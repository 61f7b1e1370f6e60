// Operand element types of the tensor-core contractions and their conversions.
//
// A tensor-core operand is stored as one plane of FP16, BF16 or TF32 (an FP32 word whose
// low 13 mantissa bits are zero), or as two planes hi + lo of the same type with
// hi = rnd(x) and lo = rnd(x - hi) ("x3" precisions: three products hi*hi + hi*lo + lo*hi).
// FP32 operands (the CUDA-core paths) are stored unrounded.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "srp_internal.h"

namespace srp {

struct tf32_t {  // FP32 storage of a TF32-rounded value
  float v;
};

// Round to TF32 (10 explicit mantissa bits), to nearest with ties away from zero.
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

template <typename T>
__device__ __forceinline__ T op_cvt(float v);
template <>
__device__ __forceinline__ float op_cvt<float>(float v) { return v; }
template <>
__device__ __forceinline__ __half op_cvt<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 op_cvt<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ tf32_t op_cvt<tf32_t>(float v) { return tf32_t{tf32_rna(v)}; }

template <typename T>
__device__ __forceinline__ float op_val(T v);
template <>
__device__ __forceinline__ float op_val<float>(float v) { return v; }
template <>
__device__ __forceinline__ float op_val<__half>(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ float op_val<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float op_val<tf32_t>(tf32_t v) { return v.v; }

// hi[idx] = rnd(v); with SPLIT also lo[idx] = rnd(v - hi).  The FP32 remainder of an FP16,
// BF16 or TF32 rounding is exact.
template <typename T, bool SPLIT>
__device__ __forceinline__ void op_store(void* hi, void* lo, size_t idx, float v) {
  const T h = op_cvt<T>(v);
  static_cast<T*>(hi)[idx] = h;
  if constexpr (SPLIT) static_cast<T*>(lo)[idx] = op_cvt<T>(v - op_val<T>(h));
}

// As above from an FP64 value (plan-time operands): the remainder is taken in FP64.
template <typename T, bool SPLIT>
__device__ __forceinline__ void op_store_d(void* hi, void* lo, size_t idx, double v) {
  const T h = op_cvt<T>(static_cast<float>(v));
  static_cast<T*>(hi)[idx] = h;
  if constexpr (SPLIT)
    static_cast<T*>(lo)[idx] = op_cvt<T>(static_cast<float>(v - static_cast<double>(op_val<T>(h))));
}

template <typename T, bool S>
struct OpTag {
  using type = T;
  static constexpr bool split = S;
};

// Calls fn(OpTag<element type, split>{}) for the operand type t (host side, e.g. to launch
// the matching kernel instantiation).
template <class Fn>
inline void op_dispatch(OpType t, Fn&& fn) {
  switch (t) {
    case OpType::F32: fn(OpTag<float, false>{}); break;
    case OpType::F16: fn(OpTag<__half, false>{}); break;
    case OpType::BF16: fn(OpTag<__nv_bfloat16, false>{}); break;
    case OpType::F16X2: fn(OpTag<__half, true>{}); break;
    case OpType::BF16X2: fn(OpTag<__nv_bfloat16, true>{}); break;
    case OpType::TF32: fn(OpTag<tf32_t, false>{}); break;
    case OpType::TF32X2: fn(OpTag<tf32_t, true>{}); break;
  }
}

}  // namespace srp
