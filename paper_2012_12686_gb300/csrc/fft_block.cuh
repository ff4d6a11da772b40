// Block-wide complex64 2-D FFT with the wavefield resident in shared memory.
//
// One CTA owns one N x N field (N = 8..128), stored row-major in shared
// memory with a leading dimension LD = N + 1 (conflict-free for both the
// row-mapped and the column-mapped passes below).  A 1-D transform of length
// N = N1 * N2 is split into two in-place Cooley-Tukey stages; the data of a
// task (one radix-N1 or radix-N2 sub-transform of one line) live in
// registers between its load and store.
//
// Along one axis, with t the task index on a line:
//   S1 (forward, radix N1, t < N2): v[i] = A[N2*i + t]  -> DFT_N1 -> * W_N^(s t k)
//                                   -> A[N2*k + t]
//   S2 (forward, radix N2, t < N1): v[i] = A[N2*t + i]  -> DFT_N2
//                                   -> v[i] holds frequency t + N1*i
//   S3 (inverse-side first stage, radix N2, t < N1): input v[i] = frequency
//        t + N1*i (exactly S2's output), DFT_N2 -> * W_N^(s t k) -> A[N2*t + k]
//   S4 (inverse-side second stage, radix N1, t < N2): v[i] = A[N2*i + t]
//        -> DFT_N1 -> v[k] holds sample N2*k + t (natural order, in place)
// S2 -> S3 and S4 -> S1 touch the same slots with the same task, so those
// pairs fuse in registers.  A propagation step F^-1{F[.] H} over both axes
// therefore costs six shared-memory round trips:
//   C14 (cols: S4 | spatial op | S1), C2, R1, R23 (rows: S2 | freq op | S3),
//   R4, C3
// and the field is in natural spatial order in shared memory between steps.
// After C2, smem row r holds y-frequency  r / N2 + N1 * (r % N2).
//
// Twiddles W_N^m = exp(-2 pi i m / N) come from a table built in FP64 on the
// host and rounded once to FP32 (at N = 128 rearranged per stage so that a task
// reads two of them per 128-bit shared load); the in-register DFT_R (R <= 16)
// uses compile-time constants of exp(+-2 pi i k / 16).
#pragma once
#include <cuda_runtime.h>
#include <utility>

namespace adorym {

// Complex arithmetic.  With ADORYM_PACKED_F32X2 (default) the real and imaginary parts go through
// the packed two-lane FP32 instructions of sm_100+ (__fadd2_rn, __fmul2_rn, __ffma2_rn): one
// instruction per complex add, two per complex multiply.  Measured on the 128 x 128 multislice
// launch: 1.32 ms packed against 1.53 ms scalar (678 M against 887 M instructions; the scalar form
// needs more registers and spills inside the passes), although in an isolated loop of transforms
// with no pointwise work the scalar form ran 5 % faster.  Every lane rounds exactly as the scalar
// form does (a - b as fma(b, -1, a), the products in the same order), so both forms give bitwise
// the same results.
#ifndef ADORYM_PACKED_F32X2
#define ADORYM_PACKED_F32X2 1
#endif
#if ADORYM_PACKED_F32X2
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return __ffma2_rn(make_float2(a.x, a.x), b, __fmul2_rn(make_float2(a.y, a.y), make_float2(-b.y, b.x)));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return __ffma2_rn(a, make_float2(b.x, b.x), __fmul2_rn(make_float2(a.y, -a.x), make_float2(b.y, b.y)));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
#else
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
#endif
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// cos / sin of 2 pi q / 32 from the first-octant values cos(2 pi j / 32), j = 0..8, by symmetry
struct Unit32 {
  static constexpr double base[9] = {1.0, 0.98078528040323044913, 0.92387953251128675613, 0.83146961230254523708,
                                     0.70710678118654752440, 0.55557023301960222474, 0.38268343236508977173,
                                     0.19509032201612826785, 0.0};
  static constexpr double cosq(int q) {   // q in [0, 32)
    return q <= 8 ? base[q] : q <= 16 ? -base[16 - q] : q <= 24 ? -base[q - 16] : base[32 - q];
  }
  static constexpr double sinq(int q) { return cosq((q + 24) % 32); }   // sin x = cos(x - pi/2)
};

// a * exp(S * 2 pi i K / R), K, R compile-time, R | 32
template <int R, int K, int S>
__device__ __forceinline__ float2 rot_const(float2 a) {
  constexpr int k = K % R;
  if constexpr (k == 0) {
    return a;
  } else if constexpr (2 * k == R) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (4 * k == R) {  // exp(S i pi/2) = S i
    return S > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
  } else if constexpr (4 * k == 3 * R) {  // exp(S i 3pi/2) = -S i
    return S > 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
  } else {
    constexpr int q = k * (32 / R);
    constexpr float c = (float)Unit32::cosq(q);
    constexpr float s = S > 0 ? (float)Unit32::sinq(q) : -(float)Unit32::sinq(q);
#if ADORYM_PACKED_F32X2
    return __ffma2_rn(make_float2(a.x, a.x), make_float2(c, s), __fmul2_rn(make_float2(a.y, a.y), make_float2(-s, c)));
#else
    return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
#endif
  }
}

template <int R, int S, int... K>
__device__ __forceinline__ void butterflies(float2 (&v)[R], const float2 (&e)[R / 2], const float2 (&o)[R / 2],
                                            std::integer_sequence<int, K...>) {
  ((v[K] = cadd(e[K], rot_const<R, K, S>(o[K])), v[K + R / 2] = csub(e[K], rot_const<R, K, S>(o[K]))), ...);
}

// In-register DFT of size R (1, 2, 4, 8, 16, 32): v[k] <- sum_n v[n] exp(S 2 pi i n k / R)
template <int R, int S>
__device__ __forceinline__ void dft(float2 (&v)[R]) {
  if constexpr (R == 1) {
    return;
  } else if constexpr (R == 2) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else {
    constexpr int H = R / 2;
    float2 e[H], o[H];
#pragma unroll
    for (int i = 0; i < H; ++i) {
      e[i] = v[2 * i];
      o[i] = v[2 * i + 1];
    }
    dft<H, S>(e);
    dft<H, S>(o);
    butterflies<R, S>(v, e, o, std::make_integer_sequence<int, H>{});
  }
}

// twiddle multiply v[k] *= W_N^(S t k) from the FP64-built table tw[m] = exp(-2 pi i m / N)
template <int S, int R>
__device__ __forceinline__ void twiddle(float2 (&v)[R], const float2* __restrict__ tw, int t) {
#pragma unroll
  for (int k = 1; k < R; ++k) {
    const float2 w = tw[t * k];
    v[k] = S < 0 ? cmul(v[k], w) : cmulc(v[k], w);
  }
}

// Twiddles of one task from a per-stage table row: row[k] = W_N^(t k), k < R (row 16-byte
// aligned), read two at a time; row[0] = 1 is skipped.  Same values as twiddle() above.
template <int S, int R>
__device__ __forceinline__ void twiddle_row(float2 (&v)[R], const float2* __restrict__ row) {
  const float4* r4 = reinterpret_cast<const float4*>(row);
#pragma unroll
  for (int k2 = 0; k2 < R / 2; ++k2) {
    const float4 w = r4[k2];
    if (k2 > 0) v[2 * k2] = S < 0 ? cmul(v[2 * k2], make_float2(w.x, w.y)) : cmulc(v[2 * k2], make_float2(w.x, w.y));
    v[2 * k2 + 1] = S < 0 ? cmul(v[2 * k2 + 1], make_float2(w.z, w.w)) : cmulc(v[2 * k2 + 1], make_float2(w.z, w.w));
  }
}

template <int N_>
struct Geo;
// NT threads per CTA; MINB resident CTAs per SM the register budget is sized for (128 regs/thread)
// The spatial passes (S4/S1, radix N1) carry the global-memory traffic of the pointwise ops, so
// N1 is the smaller radix where the two differ.
#ifndef ADORYM_NT128
#define ADORYM_NT128 512
#endif
// ADORYM_FOURPASS64: N = 64 fused kernels on the four-pass scheme of fft_block4.cuh (256 threads).
// Off by default: its radix-16 stages raised the full-size tomography probe-gradient error above
// the stored FP32 floor (1.68e-3 against a bar of 1.58e-3; the radix-8 stages of the default form
// give 1.49e-3), and the one tomography launch measured with it (scalar arithmetic) took 1.35 ms
// against 1.22 ms for the packed six-pass form of the time.
#ifndef ADORYM_FOURPASS64
#define ADORYM_FOURPASS64 0
#endif
#ifndef ADORYM_NT64
#define ADORYM_NT64 (ADORYM_FOURPASS64 ? 256 : 512)
#endif
template <> struct Geo<8>   { static constexpr int N1 = 4, N2 = 2,  NT = 64,  MINB = 8; };
template <> struct Geo<16>  { static constexpr int N1 = 4, N2 = 4,  NT = 64,  MINB = 8; };
template <> struct Geo<32>  { static constexpr int N1 = 4, N2 = 8,  NT = 128, MINB = 4; };
template <> struct Geo<64>  { static constexpr int N1 = 8, N2 = 8,  NT = ADORYM_NT64, MINB = 512 / ADORYM_NT64; };
template <> struct Geo<128> { static constexpr int N1 = 8, N2 = 16, NT = ADORYM_NT128, MINB = 1; };

template <int N>
struct Field {
  static constexpr int N1 = Geo<N>::N1, N2 = Geo<N>::N2, NT = Geo<N>::NT, LD = N + 1;
  static constexpr int SMEM_FLOAT2 = N * LD;
  // shared twiddle tables at tw (16-byte aligned): tw[m] = W_N^m (m < N); at N = 128 also the
  // S1/S4-side table [N2][N1] at tw + N and the S3-side table [N1][N2] at tw + 2N (entries
  // W_N^(t k)), which the passes read two twiddles per access (fewer shared-memory instructions,
  // -2 % time); at N = 64 the single-twiddle reads of tw measured faster
  static constexpr bool PAIRED_TW = N >= 128;
  static constexpr int TW_ENTRIES = PAIRED_TW ? 3 * N : N;
  __device__ static __forceinline__ void fill_twiddles(float2* tw, const float2* __restrict__ twg) {
    for (int i = threadIdx.x; i < N; i += NT) {
      tw[i] = twg[i];
      if (PAIRED_TW) {
        tw[N + i] = twg[(i / N1) * (i % N1)];
        tw[2 * N + i] = twg[(i / N2) * (i % N2)];
      }
    }
  }
  // y-frequency held by smem row r after the column forward stages (C2)
  __device__ static __forceinline__ int row_freq(int r) { return r / N2 + N1 * (r % N2); }
};

// ---------------------------------------------------------------------------
// Passes.  Signs are compile-time: S = -1 (DFT_-), +1 (DFT_+), 0 (stage skipped).
//
// Column pass "14": tasks (x, t < N2); v[k] <-> sample y = N2*k + t.
//   pre(pa, pb, x, t): issues the task's global loads before the smem loads and S4
//   op(v, pa, pb, x, t): spatial pointwise op on natural samples
//   S1 != 0: S1 then store; S1 == 0: store natural samples; STORE = false: no store
// LOAD = false: the samples come from op (no smem read, no S4).
// ---------------------------------------------------------------------------
struct NoPre {
  template <int R>
  __device__ __forceinline__ void operator()(float2 (&)[R], float2 (&)[R], int, int) const {}
};

// Every pass below gives each thread TPT = ceil(tasks / NT) tasks and processes them in three
// phases -- issue all loads, compute, issue all stores -- so a warp keeps several shared/global
// loads in flight instead of waiting on each task in turn (the tasks of a pass touch disjoint
// slots, so reordering them within a thread is safe).
template <int TASKS, int NT>
struct Tpt {
  static constexpr int n = (TASKS + NT - 1) / NT;
  __device__ static __forceinline__ bool ok(int tau) { return TASKS % NT == 0 || tau < TASKS; }
};

template <int N, int S4, int S1, bool LOAD, bool STORE, class Pre, class Op>
__device__ __forceinline__ void pass_c14(float2* __restrict__ A, const float2* __restrict__ tw, Pre pre, Op op) {
  using F = Field<N>;
  constexpr int N1 = F::N1, N2 = F::N2, LD = F::LD;
  using P = Tpt<N * N2, F::NT>;
  // the spatial pass keeps three register arrays per task; phase its tasks only when they fit
  constexpr int Q = (F::NT <= 512) ? (P::n < 2 ? P::n : 2) : 1;
  for (int q0 = 0; q0 < P::n; q0 += Q) {
    float2 pa[Q][N1], pb[Q][N1], v[Q][N1];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int tau = threadIdx.x + (q0 + q) * F::NT;
      if (!P::ok(tau)) continue;
      const int x = tau % N, t = tau / N;
      pre(pa[q], pb[q], x, t);
      if (LOAD) {
#pragma unroll
        for (int i = 0; i < N1; ++i) v[q][i] = A[(N2 * i + t) * LD + x];
      }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int tau = threadIdx.x + (q0 + q) * F::NT;
      if (!P::ok(tau)) continue;
      const int x = tau % N, t = tau / N;
      if (LOAD && S4) dft<N1, S4>(v[q]);
      op(v[q], pa[q], pb[q], x, t);
      if (STORE && S1) {
        dft<N1, S1>(v[q]);
        if constexpr (F::PAIRED_TW) twiddle_row<S1, N1>(v[q], tw + N + t * N1);
        else twiddle<S1>(v[q], tw, t);
      }
    }
    if (STORE) {
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int tau = threadIdx.x + (q0 + q) * F::NT;
        if (!P::ok(tau)) continue;
        const int x = tau % N, t = tau / N;
#pragma unroll
        for (int i = 0; i < N1; ++i) A[(N2 * i + t) * LD + x] = v[q][i];
      }
    }
  }
}

// Column pass "2" (S2, forward second stage) or "3" (S3, inverse-side first stage), in place.
template <int N, bool IS_S3, int S>
__device__ __noinline__ void pass_c23(float2* __restrict__ A, const float2* __restrict__ tw) {
  using F = Field<N>;
  constexpr int N1 = F::N1, N2 = F::N2, LD = F::LD;
  using P = Tpt<N * N1, F::NT>;
  float2 v[P::n][N2];
#pragma unroll
  for (int q = 0; q < P::n; ++q) {
    const int tau = threadIdx.x + q * F::NT;
    if (!P::ok(tau)) continue;
    const int x = tau % N, t = tau / N;
#pragma unroll
    for (int i = 0; i < N2; ++i) v[q][i] = A[(N2 * t + i) * LD + x];
  }
#pragma unroll
  for (int q = 0; q < P::n; ++q) {
    const int tau = threadIdx.x + q * F::NT;
    if (!P::ok(tau)) continue;
    const int t = tau / N;
    dft<N2, S>(v[q]);
    if constexpr (IS_S3) {
      if constexpr (F::PAIRED_TW) twiddle_row<S, N2>(v[q], tw + 2 * N + t * N2);
      else twiddle<S>(v[q], tw, t);
    }
  }
#pragma unroll
  for (int q = 0; q < P::n; ++q) {
    const int tau = threadIdx.x + q * F::NT;
    if (!P::ok(tau)) continue;
    const int x = tau % N, t = tau / N;
#pragma unroll
    for (int i = 0; i < N2; ++i) A[(N2 * t + i) * LD + x] = v[q][i];
  }
}

// Row pass "1" (S1 forward first stage) or "4" (S4 inverse-side second stage), in place.
template <int N, bool IS_S1, int S>
__device__ __noinline__ void pass_r14(float2* __restrict__ A, const float2* __restrict__ tw) {
  using F = Field<N>;
  constexpr int N1 = F::N1, N2 = F::N2, LD = F::LD;
  using P = Tpt<N * N2, F::NT>;
  float2 v[P::n][N1];
#pragma unroll
  for (int q = 0; q < P::n; ++q) {
    const int tau = threadIdx.x + q * F::NT;
    if (!P::ok(tau)) continue;
    const int r = tau % N, t = tau / N;
#pragma unroll
    for (int i = 0; i < N1; ++i) v[q][i] = A[r * LD + N2 * i + t];
  }
#pragma unroll
  for (int q = 0; q < P::n; ++q) {
    const int tau = threadIdx.x + q * F::NT;
    if (!P::ok(tau)) continue;
    const int t = tau / N;
    dft<N1, S>(v[q]);
    if constexpr (IS_S1) {
      if constexpr (F::PAIRED_TW) twiddle_row<S, N1>(v[q], tw + N + t * N1);
      else twiddle<S>(v[q], tw, t);
    }
  }
#pragma unroll
  for (int q = 0; q < P::n; ++q) {
    const int tau = threadIdx.x + q * F::NT;
    if (!P::ok(tau)) continue;
    const int r = tau % N, t = tau / N;
#pragma unroll
    for (int i = 0; i < N1; ++i) A[r * LD + N2 * i + t] = v[q][i];
  }
}

// Row pass "23": tasks (row r, t < N1).  Frequencies: ky = row_freq(r), kx = t + N1*i.
//   S2 != 0: smem read + S2; S2 == 0: the values come from op
//   op(v, ky, t): frequency-domain pointwise op
//   S3 != 0: S3 and store in place; S3 == 0: no store
template <int N, int S2, int S3, class Op>
__device__ __forceinline__ void pass_r23(float2* __restrict__ A, const float2* __restrict__ tw, Op op) {
  using F = Field<N>;
  constexpr int N1 = F::N1, N2 = F::N2, LD = F::LD;
  using P = Tpt<N * N1, F::NT>;
  float2 v[P::n][N2];
  if (S2) {
#pragma unroll
    for (int q = 0; q < P::n; ++q) {
      const int tau = threadIdx.x + q * F::NT;
      if (!P::ok(tau)) continue;
      const int r = tau % N, t = tau / N;
#pragma unroll
      for (int i = 0; i < N2; ++i) v[q][i] = A[r * LD + N2 * t + i];
    }
  }
#pragma unroll
  for (int q = 0; q < P::n; ++q) {
    const int tau = threadIdx.x + q * F::NT;
    if (!P::ok(tau)) continue;
    const int r = tau % N, t = tau / N;
    if (S2) dft<N2, S2>(v[q]);
    op(v[q], F::row_freq(r), t);
    if (S3) {
      dft<N2, S3>(v[q]);
      if constexpr (F::PAIRED_TW) twiddle_row<S3, N2>(v[q], tw + 2 * N + t * N2);
      else twiddle<S3>(v[q], tw, t);
    }
  }
  if (S3) {
#pragma unroll
    for (int q = 0; q < P::n; ++q) {
      const int tau = threadIdx.x + q * F::NT;
      if (!P::ok(tau)) continue;
      const int r = tau % N, t = tau / N;
#pragma unroll
      for (int i = 0; i < N2; ++i) A[r * LD + N2 * t + i] = v[q][i];
    }
  }
}

}  // namespace adorym
