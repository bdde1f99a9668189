// Device helpers shared by the render kernels.
//
// Projection (Sec. 3.1, Listing "basic"): clip = M (x, y, z, 1)^T with M
// row-major; each clip row is summed left to right, every product and sum a
// separately rounded float32 operation (__fmul_rn / __fadd_rn never fuse into
// an FMA), the division is IEEE (__fdiv_rn).  The point is culled unless
// w > 0 and finite, and unless 0 <= s < size on both axes with
// s = (clip / w * 0.5 + 0.5) * size.  pixel = floor(sx) + floor(sy) * width.
//
// Two forms here compute the same results with fewer instructions:
// - ndc * 0.5 + 0.5 is one fused multiply-add.  ndc * 0.5 is exact unless
//   |ndc| < 2^-125, and then both forms round to 0.5.
// - The tests are integer compares of bit patterns.  w lies in (0, inf)
//   exactly when bits(w) - 1 < 0x7F7FFFFF: -0, negatives and NaNs fail.  For
//   s, 0 <= s < size exactly when bits(s) < bits(size): s is never -0, and
//   negatives and NaNs have larger patterns.
// The projection has no branch: every slot of a chunk is projected, and
// culled slots drop out at the one visibility test.  The compiler can then
// interleave the divisions of a lane's slots.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pcr {

constexpr uint32_t kFullMask = 0xFFFFFFFFu;
constexpr uint32_t kNoPixel = 0xFFFFFFFFu;  // viewport is at most 16384^2 < 2^32
constexpr unsigned long long kEmptyKey = 0xFFFFFFFFFFFFFFFFull;
constexpr uint32_t kInfBits = 0x7F800000u;

// Rows 0, 1 and 3 of the matrix plus the viewport, passed by value so every
// thread reads them from the constant bank.
struct ViewParams {
  float r0[4];
  float r1[4];
  float r3[4];
  float fw, fh;
  uint32_t width;
  uint32_t height;
};

__device__ __forceinline__ float row_dot(const float r[4], float x, float y, float z) {
  return __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(r[0], x), __fmul_rn(r[1], y)), __fmul_rn(r[2], z)), r[3]);
}

__device__ __forceinline__ float to_screen(float c, float w, float size) {
  return __fmul_rn(__fmaf_rn(__fdiv_rn(c, w), 0.5f, 0.5f), size);
}

// Returns true and the pixel/depth when the point is visible.
__device__ __forceinline__ bool project(const ViewParams& v, float x, float y, float z, uint32_t& pixel,
                                        float& w) {
  w = row_dot(v.r3, x, y, z);
  const bool w_ok = __float_as_uint(w) - 1u < 0x7F7FFFFFu;
  const float cx = row_dot(v.r0, x, y, z);
  const float cy = row_dot(v.r1, x, y, z);
  const float sx = to_screen(cx, w, v.fw);
  const float sy = to_screen(cy, w, v.fh);
  if (!(w_ok && __float_as_uint(sx) < __float_as_uint(v.fw) && __float_as_uint(sy) < __float_as_uint(v.fh)))
    return false;
  // 0 <= s < size here, so converting with round-toward-minus-infinity is floor
  pixel = __float2uint_rd(sx) + __float2uint_rd(sy) * v.width;
  return true;
}

// 16-byte point load that streams past L1 and marks the line first for
// eviction in L2, so the point stream does not push the framebuffer out.
// The point buffer is read-only while a kernel runs, so the load is a pure
// function of its address and the compiler may schedule it freely.
__device__ __forceinline__ uint4 load_point_stream(const uint4* p, uint64_t policy) {
  uint4 r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
      : "l"(p), "l"(policy));
  return r;
}

__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Unsynchronised read of a framebuffer word for the early depth test
// (Sec. 3.2).  A relaxed load is not a data race against the atomics; a
// stale value can only be larger than the current one (values only
// decrease), which costs an extra atomic and never a wrong pixel.  These
// reads and the atomics below are volatile (kept in program order among
// themselves) but carry no memory clobber: nothing in a render kernel reads
// the framebuffer through ordinary loads.
__device__ __forceinline__ unsigned long long load_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ uint32_t load_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

// Fire-and-forget atomic minimum / add (the result is never read), with an
// L2 evict-last hint so the framebuffer stays resident.
__device__ __forceinline__ void red_min_u64(unsigned long long* p, unsigned long long v, uint64_t policy) {
  asm volatile("red.relaxed.gpu.global.min.u64.L2::cache_hint [%0], %1, %2;" ::"l"(p), "l"(v), "l"(policy));
}

__device__ __forceinline__ void red_min_u32(uint32_t* p, uint32_t v, uint64_t policy) {
  asm volatile("red.relaxed.gpu.global.min.u32.L2::cache_hint [%0], %1, %2;" ::"l"(p), "r"(v), "l"(policy));
}

__device__ __forceinline__ void red_add_u64(unsigned long long* p, unsigned long long v, uint64_t policy) {
  asm volatile("red.relaxed.gpu.global.add.u64.L2::cache_hint [%0], %1, %2;" ::"l"(p), "l"(v), "l"(policy));
}

// Atomic add that returns the previous value (needed by the single-atomic
// high-quality pass to detect a full primary word).
__device__ __forceinline__ unsigned long long atom_add_u64(unsigned long long* p, unsigned long long v,
                                                           uint64_t policy) {
  unsigned long long old;
  asm volatile("atom.relaxed.gpu.global.add.u64.L2::cache_hint %0, [%1], %2, %3;"
               : "=l"(old)
               : "l"(p), "l"(v), "l"(policy));
  return old;
}

__device__ __forceinline__ unsigned long long atom_exch_u64(unsigned long long* p, unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.relaxed.gpu.global.exch.b64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v));
  return old;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

}  // namespace pcr
