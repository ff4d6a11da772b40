// Block-wide complex64 N x N FFT in four shared-memory passes per propagation step (N = 128, and
// N = 64 with ADORYM_FOURPASS64; by default N = 64 takes the six-pass column passes with a row
// pass in a warp, at the end of this file, also four passes).
//
// The field is stored row-major in shared memory with leading dimension LD = N + 1, as in
// fft_block.cuh, and each 1-D transform uses the same two-stage Cooley-Tukey split (stages S1..S4
// defined there), but with different radices per axis so that two of the six passes of a
// propagation step merge.  At N = 128:
//   y: 128 = 16 * 8   (NY1 = 16: S1/S4 radix 16, stride 8;  NY2 = 8:  S2/S3 radix 8, contiguous)
//   x: 128 = 4 * 32   (NX1 = 4:  S1/S4 radix 4, stride 32;  NX2 = 32: S2/S3 radix 32, contiguous)
// With 512 threads per CTA the passes are
//   A  (x, t < 8), two tasks per thread:  y-S4 | spatial op | y-S1    samples y = 8 k + t, k < 16
//   B  (ty < 16, tx < 32):                y-S2, then x-S1             rows 8 ty + iy (iy < 8) x
//                                                                     columns 32 ix + tx (ix < 4)
//   C  (row r, t < 4):                    x-S2 | frequency op | x-S3  32 contiguous columns 32 t + i
//   B3 (ty, tx):                          x-S4, then y-S3             the slots of B
// so a propagation step F^-1{F[.] H} is A, B, C, B3 (four round trips, four barriers) instead of
// six.  Pass A, which carries the global traffic of the pointwise ops (transmission, checkpoints,
// object-gradient atomics), keeps 16 values per task; the 32-value passes B, C and B3 touch only
// shared memory, except C's frequency ops at a position's first and last transform.  After B,
// shared row r holds y-frequency r / 8 + 16 (r % 8); in C the x-frequency of element i of task t
// is t + 4 i.  Every pass reads and writes only its own slots, so one barrier follows it.
//
// At N = 64 the splits are y: 16 * 4, x: 4 * 16 with 256 threads, one task per thread in every
// pass.  Twiddles W_N^m = exp(-2 pi i m / N) come from the FP64-built table; every stage's twiddle
// index t k stays below N.
#pragma once
#include "fft_block.cuh"

namespace adorym {

template <int N_>
struct G4;
template <>
struct G4<128> {
  static constexpr int N = 128, LD = N + 1, NT = 512;
  static constexpr int NY1 = 16, NY2 = 8, NX1 = 4, NX2 = 32;
  // y-frequency held by shared row r after pass B
  __device__ static __forceinline__ int row_freq(int r) { return r / NY2 + NY1 * (r % NY2); }
};
template <>
struct G4<64> {
  static constexpr int N = 64, LD = N + 1, NT = 256;
  static constexpr int NY1 = 16, NY2 = 4, NX1 = 4, NX2 = 16;
  __device__ static __forceinline__ int row_freq(int r) { return r / NY2 + NY1 * (r % NY2); }
};

// Pass A: tasks (x, t < NY2), v[k] <-> sample y = NY2 k + t of column x; at N = 128 two tasks
// per thread, one after the other (their pointwise ops keep three 16-value arrays each).
//   pre(pa, pb, x, t): issues the task's global loads (before its shared loads and y-S4)
//   op(v, pa, pb, x, t): spatial pointwise op on natural samples
//   LOAD = false: the samples come from op (no shared read, no y-S4)
//   S1 != 0: y-S1 and store; S1 == 0: store natural samples; STORE = false: no store
template <class F4, int S4, int S1, bool LOAD, bool STORE, class Pre, class Op>
__device__ __forceinline__ void pass4_a(float2* __restrict__ A, const float2* __restrict__ tw, Pre pre, Op op) {
  constexpr int N = F4::N, LD = F4::LD, NY1 = F4::NY1, NY2 = F4::NY2, Q = (N * NY2) / F4::NT;
  static_assert(Q * F4::NT == N * NY2, "whole tasks per thread");
#pragma unroll 1
  for (int q = 0; q < Q; ++q) {
    const int tau = threadIdx.x + q * F4::NT, x = tau % N, t = tau / N;
    float2 pa[NY1], pb[NY1], v[NY1];
    pre(pa, pb, x, t);
    if (LOAD) {
#pragma unroll
      for (int i = 0; i < NY1; ++i) v[i] = A[(NY2 * i + t) * LD + x];
      if (S4) dft<NY1, S4>(v);
    }
    op(v, pa, pb, x, t);
    if (STORE) {
      if (S1) {
        dft<NY1, S1>(v);
        twiddle<S1>(v, tw, t);
      }
#pragma unroll
      for (int i = 0; i < NY1; ++i) A[(NY2 * i + t) * LD + x] = v[i];
    }
  }
}

// Pass B: y-S2 (sign SY) then x-S1 (sign SX, with its twiddles).  Task (ty < N / NY2, tx < NX2)
// holds u[iy][ix] = A[(NY2 ty + iy) LD + NX2 ix + tx].
template <class F4, int SY, int SX>
__device__ __noinline__ void pass4_b(float2* __restrict__ A, const float2* __restrict__ tw) {
  constexpr int LD = F4::LD, NY2 = F4::NY2, NX1 = F4::NX1, NX2 = F4::NX2;
  static_assert((F4::N / NY2) * NX2 == F4::NT, "one task per thread");
  const int tx = threadIdx.x % NX2, ty = threadIdx.x / NX2;
  float2 u[NY2][NX1];
#pragma unroll
  for (int iy = 0; iy < NY2; ++iy)
#pragma unroll
    for (int ix = 0; ix < NX1; ++ix) u[iy][ix] = A[(NY2 * ty + iy) * LD + NX2 * ix + tx];
#pragma unroll
  for (int ix = 0; ix < NX1; ++ix) {
    float2 c[NY2];
#pragma unroll
    for (int iy = 0; iy < NY2; ++iy) c[iy] = u[iy][ix];
    dft<NY2, SY>(c);
#pragma unroll
    for (int iy = 0; iy < NY2; ++iy) u[iy][ix] = c[iy];
  }
#pragma unroll
  for (int iy = 0; iy < NY2; ++iy) {
    dft<NX1, SX>(u[iy]);
    twiddle<SX>(u[iy], tw, tx);
  }
#pragma unroll
  for (int iy = 0; iy < NY2; ++iy)
#pragma unroll
    for (int ix = 0; ix < NX1; ++ix) A[(NY2 * ty + iy) * LD + NX2 * ix + tx] = u[iy][ix];
}

// Pass B3: x-S4 (sign SX) then y-S3 (sign SY, with its twiddles), on the slots of pass B.
template <class F4, int SX, int SY>
__device__ __noinline__ void pass4_b3(float2* __restrict__ A, const float2* __restrict__ tw) {
  constexpr int LD = F4::LD, NY2 = F4::NY2, NX1 = F4::NX1, NX2 = F4::NX2;
  static_assert((F4::N / NY2) * NX2 == F4::NT, "one task per thread");
  const int tx = threadIdx.x % NX2, ty = threadIdx.x / NX2;
  float2 u[NY2][NX1];
#pragma unroll
  for (int iy = 0; iy < NY2; ++iy)
#pragma unroll
    for (int ix = 0; ix < NX1; ++ix) u[iy][ix] = A[(NY2 * ty + iy) * LD + NX2 * ix + tx];
#pragma unroll
  for (int iy = 0; iy < NY2; ++iy) dft<NX1, SX>(u[iy]);
#pragma unroll
  for (int ix = 0; ix < NX1; ++ix) {
    float2 c[NY2];
#pragma unroll
    for (int iy = 0; iy < NY2; ++iy) c[iy] = u[iy][ix];
    dft<NY2, SY>(c);
    twiddle<SY>(c, tw, ty);
#pragma unroll
    for (int iy = 0; iy < NY2; ++iy) u[iy][ix] = c[iy];
  }
#pragma unroll
  for (int iy = 0; iy < NY2; ++iy)
#pragma unroll
    for (int ix = 0; ix < NX1; ++ix) A[(NY2 * ty + iy) * LD + NX2 * ix + tx] = u[iy][ix];
}

// Pass C: task (row r, t < NX1), one per thread; v[i] = A[r LD + NX2 t + i].
//   S2 != 0: shared read + x-S2; S2 == 0: the values come from op
//   op(v, ky, t): frequency-domain op, x-frequency of v[i] is t + NX1 i
//   S3 != 0: x-S3 and store in place; S3 == 0: no store
template <class F4, int S2, int S3, class Op>
__device__ __forceinline__ void pass4_c(float2* __restrict__ A, const float2* __restrict__ tw, Op op) {
  constexpr int N = F4::N, LD = F4::LD, NX2 = F4::NX2;
  static_assert(N * F4::NX1 == F4::NT, "one task per thread");
  const int r = threadIdx.x % N, t = threadIdx.x / N;
  float2 v[NX2];
  if (S2) {
#pragma unroll
    for (int i = 0; i < NX2; ++i) v[i] = A[r * LD + NX2 * t + i];
    dft<NX2, S2>(v);
  }
  op(v, F4::row_freq(r), t);
  if (S3) {
    dft<NX2, S3>(v);
    twiddle<S3>(v, tw, t);
#pragma unroll
    for (int i = 0; i < NX2; ++i) A[r * LD + NX2 * t + i] = v[i];
  }
}

}  // namespace adorym

namespace adorym {

// The pass sequence of the fused kernels, per tile size.  Values per spatial-pass task CY at
// y = YS k + t (k < CY); values per frequency-pass task RX at x-frequency t + KXS i (i < RX).
//   c14<S4, S1, LOAD, STORE>(A, tw, pre, op)   y-S4 | spatial op | y-S1
//   fwd_pair<S>(A, tw)                         y-S2 then x-S1 (with a barrier between them
//                                              where they are separate passes)
//   r23<S2, S3>(A, tw, op)                     x-S2 | frequency op | x-S3
//   inv_pair<S>(A, tw)                         x-S4 then y-S3
// N <= 32: the six-pass scheme of fft_block.cuh; N = 64: its column passes with the row passes in
// a warp (below); N = 128: the four-pass scheme above.
template <int N>
struct PathFFT {
  using F = Field<N>;
  static constexpr int CY = F::N1, YS = F::N2, RX = F::N2, KXS = F::N1;
  template <int S4, int S1, bool LOAD, bool STORE, class Pre, class Op>
  __device__ static __forceinline__ void c14(float2* A, const float2* tw, Pre pre, Op op) {
    pass_c14<N, S4, S1, LOAD, STORE>(A, tw, pre, op);
  }
  template <int S>
  __device__ static __forceinline__ void fwd_pair(float2* A, const float2* tw) {
    pass_c23<N, false, S>(A, tw);
    __syncthreads();
    pass_r14<N, true, S>(A, tw);
  }
  template <int S2, int S3, class Op>
  __device__ static __forceinline__ void r23(float2* A, const float2* tw, Op op) {
    pass_r23<N, S2, S3>(A, tw, op);
  }
  template <int S>
  __device__ static __forceinline__ void inv_pair(float2* A, const float2* tw) {
    pass_r14<N, false, S>(A, tw);
    __syncthreads();
    pass_c23<N, true, S>(A, tw);
  }
};

template <int N>
struct PathFFT4 {
  using G = G4<N>;
  static constexpr int CY = G::NY1, YS = G::NY2, RX = G::NX2, KXS = G::NX1;
  template <int S4, int S1, bool LOAD, bool STORE, class Pre, class Op>
  __device__ static __forceinline__ void c14(float2* A, const float2* tw, Pre pre, Op op) {
    static_assert(Geo<N>::NT == G::NT, "the four-pass scheme sets the CTA's thread count");
    pass4_a<G, S4, S1, LOAD, STORE>(A, tw, pre, op);
  }
  template <int S>
  __device__ static __forceinline__ void fwd_pair(float2* A, const float2* tw) {
    pass4_b<G, S, S>(A, tw);
  }
  template <int S2, int S3, class Op>
  __device__ static __forceinline__ void r23(float2* A, const float2* tw, Op op) {
    pass4_c<G, S2, S3>(A, tw, op);
  }
  template <int S>
  __device__ static __forceinline__ void inv_pair(float2* A, const float2* tw) {
    pass4_b3<G, S, S>(A, tw);
  }
};

template <>
struct PathFFT<128> : PathFFT4<128> {};
#if ADORYM_FOURPASS64
template <>
struct PathFFT<64> : PathFFT4<64> {};
#else
// N = 64: the column passes as in the six-pass scheme, the x transforms of a step in one row pass.
// The eight tasks of a row (t < 8) are eight lanes of one warp, so the slot exchange between a
// row's two radix-8 stages (S1 -> S2 forward, S3 -> S4 inverse) goes through a per-warp scratch
// area with warp-level synchronisation instead of a shared-memory pass and a CTA barrier:
//   C14 | C2 | R (x-S1 | exchange | x-S2 | frequency op | x-S3 | exchange | x-S4) | C3
// is four passes and four barriers per propagation step instead of six, with the same stages,
// twiddles and order (the same values).  The spatial pass keeps the six-pass thread mapping
// (consecutive x across a warp: coalesced global accesses); only the row pass, which touches no
// global memory, uses the warp layout: lane 8 g + t of warp w holds task t of row
// (w & 7) + 8 g + 32 (w >> 3), so the two rows of a half-warp differ by 8 and every 64-bit row
// access of a warp covers all 32 banks at leading dimension 65.
// Exchange: lane (g, a) stores its value k at scratch[72 g + a + 9 k]; lane (g, b) reads its
// value i from scratch[72 g + i + 9 b] (both conflict-free).

// per-warp exchange scratch of the row pass: one array per CTA
__device__ __forceinline__ float2* row64_scratch() {
  __shared__ float2 scratch[(Geo<64>::NT / 32) * 288];
  return scratch;
}

template <int S>
__device__ __forceinline__ void row64_line(float2 (&v)[8], const float2 (&wt)[8], float2* __restrict__ ws, int g,
                                           int a) {
  dft<8, S>(v);
#pragma unroll
  for (int k = 1; k < 8; ++k) v[k] = S < 0 ? cmul(v[k], wt[k]) : cmulc(v[k], wt[k]);   // twiddle<S>
  __syncwarp();   // the previous exchange of this warp has read its slots
#pragma unroll
  for (int k = 0; k < 8; ++k) ws[72 * g + a + 9 * k] = v[k];
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = ws[72 * g + i + 9 * a];
  dft<8, S>(v);
}

template <>
struct PathFFT<64> {
  using F = Field<64>;
  static_assert(F::N1 == 8 && F::N2 == 8 && F::NT == 512 && !F::PAIRED_TW, "row pass layout");
  static constexpr int CY = F::N1, YS = F::N2, RX = F::N2, KXS = F::N1;
  template <int S4, int S1, bool LOAD, bool STORE, class Pre, class Op>
  __device__ static __forceinline__ void c14(float2* A, const float2* tw, Pre pre, Op op) {
    pass_c14<64, S4, S1, LOAD, STORE>(A, tw, pre, op);
  }
  template <int S>
  __device__ static __forceinline__ void fwd_pair(float2* A, const float2* tw) {
    pass_c23<64, false, S>(A, tw);
  }
  // row r (y-frequency row_freq(r)): S2 != 0 reads samples x = 8 i + t and runs x-S1, x-S2; op
  // sees x-frequencies t + 8 i; S3 != 0 runs x-S3, x-S4 and stores samples in place
  template <int S2, int S3, class Op>
  __device__ static __forceinline__ void r23(float2* A, const float2* tw, Op op) {
    constexpr int LD = F::LD;
    const int lane = (int)(threadIdx.x & 31), w = (int)(threadIdx.x >> 5), g = lane >> 3, t = lane & 7;
    const int r = (w & 7) + 8 * g + 32 * (w >> 3);
    float2* ws = row64_scratch() + w * 288;
    float2 v[8], wt[8];
#pragma unroll
    for (int k = 1; k < 8; ++k) wt[k] = tw[t * k];
    if (S2) {
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] = A[r * LD + 8 * i + t];
      row64_line<S2>(v, wt, ws, g, t);
    }
    op(v, F::row_freq(r), t);
    if (S3) {
      row64_line<S3>(v, wt, ws, g, t);
#pragma unroll
      for (int k = 0; k < 8; ++k) A[r * LD + 8 * k + t] = v[k];
    }
  }
  template <int S>
  __device__ static __forceinline__ void inv_pair(float2* A, const float2* tw) {
    pass_c23<64, true, S>(A, tw);
  }
};
#endif

}  // namespace adorym
