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
//
// project_pair computes the same results for two slots at once (see there):
// Blackwell's paired float32 instructions (each half rounded on its own, as
// the scalar instruction rounds it) for the matrix rows and the screen
// transform, and one reciprocal per slot shared by both screen divisions,
// with Markstein's correction making each quotient the IEEE one.
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

// ---------------------------------------------------------------------------
// Two slots at once.
// ---------------------------------------------------------------------------

// Two floats in one 64-bit register pair: slot a in the low half, slot b in
// the high half.  mul/fma .rn.f32x2 round each half on its own, exactly as
// the scalar .rn instruction would (no flush to zero).
using f32x2 = unsigned long long;

__device__ __forceinline__ f32x2 f2_pack(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(f32x2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 f2_bcast(float x) { return f2_pack(x, x); }
__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

__device__ __forceinline__ float add_rn(float a, float b) {
  float r;
  asm("add.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}

// One matrix row for two slots: the three products as paired instructions,
// the sums as scalar add.rn on the halves.  Paired sums are not used: ptxas
// fuses a paired product into a following paired add (or into fma with a
// factor of one) despite the .rn modifier, which would change roundings.
// A scalar add.rn is never fused.
__device__ __forceinline__ f32x2 row_dot2(const float r[4], f32x2 x, f32x2 y, f32x2 z) {
  float a0, b0, a1, b1, a2, b2;
  f2_unpack(f2_mul(f2_bcast(r[0]), x), a0, b0);
  f2_unpack(f2_mul(f2_bcast(r[1]), y), a1, b1);
  f2_unpack(f2_mul(f2_bcast(r[2]), z), a2, b2);
  return f2_pack(add_rn(add_rn(add_rn(a0, a1), a2), r[3]), add_rn(add_rn(add_rn(b0, b1), b2), r[3]));
}

// Hardware reciprocal estimate (within 1 ulp of 1/w).
__device__ __forceinline__ float rcp_estimate(float w) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(w));
  return r;
}

// w for which the reciprocal path below is exact: [2^-40, 2^40).  Every
// quantity it forms is then a normal number or an exact zero, or the point
// is culled either way (below).
constexpr uint32_t kRcpWindowLo = 0x2B800000u;                  // bits of 2^-40
constexpr uint32_t kRcpWindowSpan = 0x53800000u - kRcpWindowLo;  // up to bits of 2^40

__device__ __forceinline__ bool in_rcp_window(float w) {
  return __float_as_uint(w) - kRcpWindowLo < kRcpWindowSpan;
}

// RN(1/w) for both halves: one Newton step with fused operations on the
// estimate y0, y1 = y0 + y0 (1 - w y0).  nw holds -w.
__device__ __forceinline__ f32x2 reciprocal2(f32x2 nw, float wa, float wb) {
  const f32x2 y0 = f2_pack(rcp_estimate(wa), rcp_estimate(wb));
  return f2_fma(y0, f2_fma(nw, y0, f2_bcast(1.0f)), y0);
}

// c / w rounded to nearest even, given y = RN(1/w) (Markstein, IBM J. Res.
// Dev. 34(1), 1990): q0 = RN(c y) lies within one ulp of c / w, so the
// remainder r = c - q0 w is exact in one fused operation, and RN(q0 + r y)
// is the correctly rounded quotient.  That holds while nothing overflows or
// underflows: for w in the window and |c / w| >= 2^-30 every term is normal
// or an exact zero.  Smaller quotients come out below 2^-27 in magnitude, and
// every such quotient gives ndc * 0.5 + 0.5 = 0.5 exactly, as the exact one
// does.  Where c y overflows (|c / w| near 2^128) the result is infinite or
// NaN, and the point is culled, as with the exact quotient (|c / w| > 2).
__device__ __forceinline__ f32x2 quotient2(f32x2 c, f32x2 nw, f32x2 y) {
  const f32x2 q0 = f2_mul(c, y);
  return f2_fma(f2_fma(q0, nw, c), y, q0);
}

// project() for slots a and b: the same results, bit for bit.  The matrix
// rows are summed in the same order with the same roundings; the screen
// transform is the same fused multiply-add and product; each quotient equals
// the IEEE one (quotient2).  A slot whose w is valid but outside the window
// takes the IEEE divisions.  pa / pb are meaningful only when va / vb.
__device__ __forceinline__ void project_pair(const ViewParams& v, const uint4& ra, const uint4& rb, uint32_t& pa,
                                             uint32_t& pb, float& wa, float& wb, bool& va, bool& vb) {
  const f32x2 x = f2_pack(__uint_as_float(ra.x), __uint_as_float(rb.x));
  const f32x2 y = f2_pack(__uint_as_float(ra.y), __uint_as_float(rb.y));
  const f32x2 z = f2_pack(__uint_as_float(ra.z), __uint_as_float(rb.z));
  const f32x2 w2 = row_dot2(v.r3, x, y, z);
  const f32x2 cx = row_dot2(v.r0, x, y, z);
  const f32x2 cy = row_dot2(v.r1, x, y, z);
  f2_unpack(w2, wa, wb);
  const f32x2 nw = f2_mul(w2, f2_bcast(-1.0f));
  const f32x2 rw = reciprocal2(nw, wa, wb);
  float sxa, sxb, sya, syb;
  f2_unpack(f2_mul(f2_fma(quotient2(cx, nw, rw), f2_bcast(0.5f), f2_bcast(0.5f)), f2_bcast(v.fw)), sxa, sxb);
  f2_unpack(f2_mul(f2_fma(quotient2(cy, nw, rw), f2_bcast(0.5f), f2_bcast(0.5f)), f2_bcast(v.fh)), sya, syb);
  const bool oka = __float_as_uint(wa) - 1u < 0x7F7FFFFFu;
  const bool okb = __float_as_uint(wb) - 1u < 0x7F7FFFFFu;
  const bool slowa = oka && !in_rcp_window(wa);
  const bool slowb = okb && !in_rcp_window(wb);
  if (slowa || slowb) {
    float cxa, cxb, cya, cyb;
    f2_unpack(cx, cxa, cxb);
    f2_unpack(cy, cya, cyb);
    if (slowa) {
      sxa = to_screen(cxa, wa, v.fw);
      sya = to_screen(cya, wa, v.fh);
    }
    if (slowb) {
      sxb = to_screen(cxb, wb, v.fw);
      syb = to_screen(cyb, wb, v.fh);
    }
  }
  const uint32_t bw = __float_as_uint(v.fw), bh = __float_as_uint(v.fh);
  va = oka && __float_as_uint(sxa) < bw && __float_as_uint(sya) < bh;
  vb = okb && __float_as_uint(sxb) < bw && __float_as_uint(syb) < bh;
  pa = __float2uint_rd(sxa) + __float2uint_rd(sya) * v.width;
  pb = __float2uint_rd(sxb) + __float2uint_rd(syb) * v.width;
}

// Every slot of a chunk: pairs, then a last single slot when U is odd.
// pix[u] is meaningful only when vis[u].
template <int U>
__device__ __forceinline__ void project_slots(const ViewParams& v, const uint4 (&r)[U], uint32_t (&pix)[U],
                                              float (&w)[U], bool (&vis)[U]) {
#pragma unroll
  for (int u = 0; u + 1 < U; u += 2)
    project_pair(v, r[u], r[u + 1], pix[u], pix[u + 1], w[u], w[u + 1], vis[u], vis[u + 1]);
  if constexpr (U % 2 == 1) {
    pix[U - 1] = 0;
    w[U - 1] = 0.0f;
    vis[U - 1] = project(v, __uint_as_float(r[U - 1].x), __uint_as_float(r[U - 1].y), __uint_as_float(r[U - 1].z),
                         pix[U - 1], w[U - 1]);
  }
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

// Two neighbouring 16-byte records (32-byte aligned) in one 32-byte load,
// with the same caching as load_point_stream.
__device__ __forceinline__ void load_pair_stream(const uint4* p, uint64_t policy, uint4& a, uint4& b) {
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], %9;"
      : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
      : "l"(p), "l"(policy));
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
