// Device-side check of the screen division the projection uses
// (common.cuh: reciprocal2, quotient2, project_pair) against the device's own
// IEEE operations.  A diagnostic behind pcr_check_division: nothing on the
// render path calls it.
//
// The projection divides both clip coordinates by w through one reciprocal
// per point, y = RN(1/w) from one Newton step on the hardware estimate, then
// corrects each quotient after Markstein (1990).  The claims checked here:
//   - y equals the IEEE reciprocal for every w in the window [2^-40, 2^40);
//   - the quotient equals IEEE c / w wherever 2^-30 <= |c / w| <= 2^126;
//   - the screen coordinate (ndc * 0.5 + 0.5) * size is bit-identical to
//     the one from the IEEE quotient, or culled on both sides, for every c.
#include <cstdint>

#include "../../include/pcr.h"
#include "common.cuh"
#include "launch.h"

namespace pcr {

namespace {

// reciprocal mismatches, quotient mismatches, screen mismatches, pairs in the
// quotient's domain, pairs checked
__device__ unsigned long long g_check_counts[5];

__device__ __forceinline__ void warp_add(unsigned long long* dst, unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFullMask, v, o);
  if (lane_id() == 0 && v != 0) atomicAdd(dst, v);
}

__global__ void k_check_reciprocal(uint32_t first, uint32_t count) {
  unsigned long long bad = 0;
  for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < count;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const float w = __uint_as_float(first + static_cast<uint32_t>(i));
    if (!in_rcp_window(w)) continue;
    float ya, yb;
    f2_unpack(reciprocal2(f2_bcast(-w), w, w), ya, yb);
    const uint32_t ref = __float_as_uint(__frcp_rn(w));
    bad += (__float_as_uint(ya) != ref) + (__float_as_uint(yb) != ref);
  }
  warp_add(&g_check_counts[0], bad);
}

__device__ __forceinline__ bool screen_culled(float s, float size) {
  return !(__float_as_uint(s) < __float_as_uint(size));
}

// Pairs (w, c): a block takes one w = w_first + i at a time, i in
// [i_first, i_end), and its threads walk the numerators c = c_bits[j] or
// c_first + j * c_step, j < c_count.
__global__ void k_check_quotient(uint32_t w_first, uint32_t i_first, uint32_t i_end, uint32_t c_count,
                                 const uint32_t* __restrict__ c_bits, uint32_t c_first, uint32_t c_step, float size) {
  unsigned long long qbad = 0, sbad = 0, qpairs = 0, pairs = 0;
  for (uint32_t i = i_first + blockIdx.x; i < i_end; i += gridDim.x) {
    const float w = __uint_as_float(w_first + i);
    if (!in_rcp_window(w)) continue;  // the projection divides exactly there
    const f32x2 nw = f2_bcast(-w);
    const f32x2 y = reciprocal2(nw, w, w);
    for (uint32_t j = threadIdx.x; j < c_count; j += blockDim.x) {
      const float c = __uint_as_float(c_bits ? c_bits[j] : c_first + j * c_step);
      ++pairs;
      float qa, qb;
      f2_unpack(quotient2(f2_bcast(c), nw, y), qa, qb);
      const float exact = __fdiv_rn(c, w);
      const float mag = fabsf(exact);
      if (mag >= 0x1p-30f && mag <= 0x1p126f) {
        ++qpairs;
        qbad += __float_as_uint(qa) != __float_as_uint(exact) || __float_as_uint(qb) != __float_as_uint(exact);
      }
      const float s_fast = __fmul_rn(__fmaf_rn(qa, 0.5f, 0.5f), size);
      const float s_exact = to_screen(c, w, size);
      const bool cf = screen_culled(s_fast, size), ce = screen_culled(s_exact, size);
      sbad += cf != ce || (!ce && __float_as_uint(s_fast) != __float_as_uint(s_exact));
    }
  }
  warp_add(&g_check_counts[1], qbad);
  warp_add(&g_check_counts[2], sbad);
  warp_add(&g_check_counts[3], qpairs);
  warp_add(&g_check_counts[4], pairs);
}

}  // namespace

cudaError_t check_division(uint32_t w_first, uint32_t w_count, const uint32_t* c_bits, uint32_t c_first,
                           uint32_t c_count, uint32_t c_step, float size, uint64_t out[5], cudaStream_t s,
                           const Device& d) {
  const unsigned long long zero[5] = {0, 0, 0, 0, 0};
  cudaError_t e = cudaMemcpyToSymbolAsync(g_check_counts, zero, sizeof(zero), 0, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  const dim3 grid(static_cast<unsigned>(d.num_sms) * 8u), block(256);
  if (w_count > 0) {
    k_check_reciprocal<<<grid, block, 0, s>>>(w_first, w_count);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // the pairs in launches of at most about 2^33 each, so no launch runs long
  if (c_count > 0) {
    const uint64_t per = (1ull << 33) / c_count;
    const uint32_t step = static_cast<uint32_t>(per < 1 ? 1 : (per > w_count ? w_count : per));
    for (uint64_t i = 0; i < w_count; i += step) {
      const uint32_t end = static_cast<uint32_t>(i + step < w_count ? i + step : w_count);
      k_check_quotient<<<grid, block, 0, s>>>(w_first, static_cast<uint32_t>(i), end, c_count, c_bits, c_first,
                                              c_step, size);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  unsigned long long got[5];
  if ((e = cudaMemcpyFromSymbolAsync(got, g_check_counts, sizeof(got), 0, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  for (int k = 0; k < 5; ++k) out[k] = got[k];
  return cudaSuccess;
}

}  // namespace pcr
