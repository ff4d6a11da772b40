// Numerical helpers that keep per-element work off the FP64 pipe.  FP64 arithmetic and
// FP32<->FP64 conversions run at a small fraction of the FP32 rate on this part, so the FP64
// reductions (object-gradient accumulators, loss sums) take their per-element steps here and use
// FP64 arithmetic only once per thread or in the memory system (double atomics at L2), and the
// sub-pixel shift ramps are formed with FP32 error-free steps instead of an FP64 reduction.
#pragma once
#include <cuda_runtime.h>

namespace adorym {

// Exact binary32 -> binary64 widening from the IEEE 754 encodings, in integer arithmetic.  With
// a = |x| as bits (biased exponent e in bits 23..30, significand m in bits 0..22), a >> 3 puts e at
// bit 20 and the top 20 significand bits below it, so adding (1023 - 127) << 20 rebiases the
// exponent; the 3 lowest significand bits become the top of the low word.  Infinities and NaNs
// (e = 255) get the rebias that lands on the all-ones exponent 2047 instead; zeros and subnormal
// inputs (|x| < 2^-126) become a signed zero (an absolute change below 1.2e-38).  About ten
// integer instructions, none on the FP64 pipe.
__device__ __forceinline__ double f32_to_f64(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned a = u & 0x7FFFFFFFu;
  const bool tiny = a < 0x00800000u;
  const unsigned bias = tiny ? 0u : (a >= 0x7F800000u ? 0x70000000u : 0x38000000u);
  const unsigned mag = tiny ? 0u : a;
  const unsigned hi = ((mag >> 3) + bias) | (u & 0x80000000u);
  const unsigned lo = mag << 29;
  return __hiloint2double((int)hi, (int)lo);
}

// binary64 -> binary32 narrowing from the IEEE 754 encodings (hi, lo = upper and lower 32 bits
// of the double), in integer arithmetic, rounding to nearest with ties to even: the top 23 of the
// 52 significand bits are kept, the 29 dropped bits decide the rounding (a carry moves into the
// exponent, and past the largest finite value gives infinity).  Magnitudes below 2^-126 become a
// signed zero (an absolute change below 1.2e-38); infinities stay infinite, NaNs become a NaN.
__device__ __forceinline__ float f64bits_to_f32(unsigned hi, unsigned lo) {
  const unsigned sign = hi & 0x80000000u;
  const unsigned ah = hi & 0x7FFFFFFFu;
  const int e = (int)(ah >> 20) - (1023 - 127);
  unsigned r = ((unsigned)max(e, 0) << 23) | ((ah & 0xFFFFFu) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1FFFFFFFu;
  r += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;
  if (e <= 0) r = 0u;
  if (e >= 255) r = (ah > 0x7FF00000u || (ah == 0x7FF00000u && lo != 0u)) ? 0x7FC00000u : 0x7F800000u;
  return __uint_as_float(sign | r);
}
__device__ __forceinline__ float f64_to_f32(const double* p) {   // load and narrow (read-only data)
  const uint2 w = __ldg(reinterpret_cast<const uint2*>(p));
  return f64bits_to_f32(w.y, w.x);
}

// Set a bit of a call's status word.  Plain read-modify-write rather than an atomic: the word may
// live in mapped host memory, and every writer within one kernel sets the same bit.
__device__ __forceinline__ void set_status(int* status, int bit) {
  volatile int* s = status;
  *s = *s | bit;
}

// Integer patch corner floor(pos + 1/2) of the position split (Sec. 2.3.1), clamped to +-2^24 so
// that corner + patch offsets and corner + N never overflow an int; a non-finite position gives
// corner 0 (the input check reports it).
__device__ __forceinline__ int patch_corner(float pos) {
  const double f = floor((double)pos + 0.5);
  return f != f ? 0 : (int)fmin(fmax(f, -16777216.0), 16777216.0);
}

// Compensated FP32 running sum (Kahan summation): the low-order part lost by each addition is
// carried in c and fed back into the next one, so the sum of n terms is accurate to a few ulps
// of sum |x_i| independent of n.  Read out once, in FP64.
struct Kahan {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return f32_to_f64(s) - f32_to_f64(c); }
};

// Fourier shift ramp exp(-2 pi i d f_k) of Eq. fourier_shift, f_k = k'/N with k' the signed
// frequency index of bin k (Nyquist bin negative), N a power of two <= 2048.  The phase in units
// of pi, -2 d k'/N, is formed without rounding: d is split into a high part with 12 significant
// bits and the exact remainder (also <= 12 bits), each product with |k'| <= 2^10 needs at most 22
// bits, the scaling by 2/N is a power of two, and removing the nearest even integer from the
// high part is exact.  The one rounding is the final addition, so the argument passed to
// sincospif is the exact phase reduced to [-1, 1] and rounded once.
__device__ __forceinline__ float2 shift_ramp(float d, int k, int N) {
  const int kk = k <= (N - 1) / 2 ? k : k - N;
  const float dh = __uint_as_float(__float_as_uint(d) & 0xFFFFF000u);
  const float dl = d - dh;
  const float sc = -2.0f / (float)N;
  float ph = (dh * (float)kk) * sc;
  const float pl = (dl * (float)kk) * sc;
  ph -= 2.0f * rintf(0.5f * ph);
  float s, c;
  sincospif(ph + pl, &s, &c);
  return make_float2(c, s);
}

}  // namespace adorym
