// Two-pass path for tiles of 256, 512 and 1024 pixels: the wavefields live in HBM and each
// propagation step is one row kernel and one column kernel.
//
// A 1-D transform of length N = N1 * N2 uses the same two in-place stages as the shared-memory
// kernel (S1/S2 forward, S3/S4 inverse side, see fft_block.cuh), so a field in global memory is
// always in natural order: spatial (y, x), or "x-transformed" (y, kx) between a row kernel and
// a column kernel.
//
//   row kernel  (RB rows per CTA):   [S3 S4 from global]  -> spatial op ->  [S1 S2 to global]
//   column kernel (CW columns/CTA):  [S1 S2 from global]  -> frequency op -> [S3 S4 to global]
//
// so one slice step (modulation by T_j, Eq. ri_modulation; Fresnel step, Eq. fresnel_prop)
// is: row kernel (finish the previous inverse x-transform, store/modulate, start the forward
// x-transform) + column kernel (forward y-transform, propagator, inverse y-transform).  The
// row tile uses a skewed shared-memory layout (one pad element after every N2 elements), which
// keeps both the strided and the contiguous stage accesses free of bank conflicts with the
// lane index on the x digit, so every global access is coalesced.  The column tile is brought in
// by TMA (a 2-D tensor map over the field buffer, completion on an mbarrier) and lands in the
// [row][column] layout the first in-place stage reads.  With one probe mode and measured data the
// detector pass also forms the loss term and the adjoint seed.  Loss and position-gradient
// reductions write per-CTA FP64 partials (compensated FP32 within a CTA) that a final kernel adds
// in a fixed order.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>

#include "numerics.cuh"
#include "fft_block.cuh"
#include "kernels.cuh"

namespace adorym {

template <int N>
struct Geo2;
// RB rows per row-kernel CTA, CW columns per column-kernel CTA; 256 threads, tiles of ~64 KB so
// two CTAs share an SM and one CTA's loads overlap the other's transforms
template <> struct Geo2<256>  { static constexpr int N1 = 16, N2 = 16, RB = 16, CW = 32; };
template <> struct Geo2<512>  { static constexpr int N1 = 16, N2 = 32, RB = 16, CW = 16; };
template <> struct Geo2<1024> { static constexpr int N1 = 32, N2 = 32, RB = 8, CW = 8; };
constexpr int NT2 = 256;

template <int N>
constexpr int row_smem_bytes() {
  return Geo2<N>::RB * (N + Geo2<N>::N1) * (int)sizeof(float2) + N * (int)sizeof(float2) + 64 * 8;
}
// column tile + tw, ry, hy tables + 64 doubles of reduction scratch + one mbarrier (TMA staging)
template <int N>
constexpr int col_smem_bytes() {
  return N * Geo2<N>::CW * (int)sizeof(float2) + 3 * N * (int)sizeof(float2) + 64 * 8 + 16;
}

// R_NEAR_DSEED / C_FAR_SEED (one probe mode with measured data; the _P forms for the Poisson loss,
// so that each kernel carries one loss's code): detector intensity, loss term and
// adjoint seed 2 dL/dI Psi in the same pass, replacing R_NEAR_DET / C_FAR + k_loss2 + R_NEAR_SEED /
// C_SEED
enum RowMode { R_FWD, R_RC_FIRST, R_RC, R_ADJ, R_NEAR_DET, R_NEAR_SEED, R_PHAT, R_PG_OUT, R_NEAR_DSEED, R_NEAR_DSEED_P };
enum ColMode { C_PROP, C_PROP_ADJ, C_PSI0, C_FAR, C_SEED, C_Q, C_PHAT, C_PG, C_NEAR_PHI, C_NEAR_Q, C_FAR_SEED, C_FAR_SEED_P };

// Resident CTAs per SM the register budget of a row / column kernel is sized for.  At N = 256 the
// slice-step kernels of the forward and recompute sweeps and the propagation column kernels fit
// three per SM without spilling (80 registers; shared memory 37 / 71 KB per CTA), which puts more
// loads in flight in these latency-bound passes; the other modes keep two (their larger register
// sets would spill).  ADORYM_TP256_OCC3 = 0 keeps two everywhere.
#ifndef ADORYM_TP256_OCC3
#define ADORYM_TP256_OCC3 1
#endif
template <int N, int MODE>
constexpr int row_minb() {
  return (ADORYM_TP256_OCC3 && N == 256 && (MODE == R_FWD || MODE == R_RC_FIRST)) ? 3 : 2;
}
template <int N, int MODE>
constexpr int col_minb() {
  return (ADORYM_TP256_OCC3 && N == 256 && (MODE == C_PROP || MODE == C_PROP_ADJ)) ? 3 : 2;
}

__device__ __forceinline__ float freqf(int k, int N) { return (float)(k <= (N - 1) / 2 ? k : k - N) / (float)N; }

// per-pixel term of Eq. lsq_loss (amplitudes, I + eps) or Eq. poisson_loss, and dL/dI before the
// 1 / npix normalisation
__device__ __forceinline__ float loss_term(int loss, float I, float im, float eps, float* dI) {
  if (loss == 0) {
    const float sI = sqrtf(I + eps), sM = sqrtf(im + eps);
    const float df = sI - sM;
    *dI = df / sI;
    return df * df;
  }
  *dI = 1.0f - im / (I + eps);
  return I - im * logf(I + eps);
}

__device__ __forceinline__ double block_sum2(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  __syncthreads();
  return s;
}

// TwoSum (Knuth): s + e == a + b exactly, in FP32
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// CTA sums of three FP32 values, in FP64 on thread 0 (out[]): a compensated warp tree (each
// level adds the high parts with TwoSum and carries the error in the low parts), then an FP64
// sum over the warps in a fixed order.  One pass for three values, no FP64 shuffles.
__device__ __forceinline__ void block_sum3(float a0, float a1, float a2, double* red, double out[3]) {
  float hi[3] = {a0, a1, a2}, lo[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float h = __shfl_xor_sync(0xffffffffu, hi[q], o), l = __shfl_xor_sync(0xffffffffu, lo[q], o);
      float sum, err;
      two_sum(hi[q], h, sum, err);
      hi[q] = sum;
      lo[q] += l + err;
    }
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0)
    for (int q = 0; q < 3; ++q) red[3 * w + q] = f32_to_f64(hi[q]) + f32_to_f64(lo[q]);
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < 3; ++q) {
      double t = 0.0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[3 * i + q];
      out[q] = t;
    }
  }
  __syncthreads();
}

// ============================================================================ TMA staging
// The column kernels' N x CW tiles are brought into shared memory by the tensor-memory
// accelerator: one thread issues min(N, 256)-row boxes of a 2-D tensor map over the field buffer
// (cp.async.bulk.tensor), completion is counted in bytes on an mbarrier, and every thread waits on
// the barrier's phase, for at most about a second (then the call's status word records the
// timeout and the CTA leaves after a second bounded wait for its copies).
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// wait for phase `phase` of the barrier for at most `limit` clock cycles (about 2^31, a second,
// by default); a negative limit reports a timeout without waiting (the test hook of the
// timeout branch: the caller then waits for its copies with the default limit before it leaves)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase, long long limit = 1LL << 31) {
  if (limit < 0) return false;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, phase))
    if (clock64() - t0 > limit) return false;
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// ============================================================================ row kernel
template <int N, int MODE>
__global__ void __launch_bounds__(NT2, row_minb<N, MODE>()) k_row(const TPArgs a) {
  constexpr int N1 = Geo2<N>::N1, N2 = Geo2<N>::N2, RB = Geo2<N>::RB, LDR = N + N1;
  constexpr size_t NN = (size_t)N * N;
  extern __shared__ float2 sm[];
  float2* A = sm;
  float2* tw = A + RB * LDR;
  double* red = reinterpret_cast<double*>(tw + N);
  auto idx = [](int r, int p) { return r * LDR + p + p / N2; };
  for (int i = threadIdx.x; i < N; i += NT2) tw[i] = a.tw[i];

  const int r0 = blockIdx.x * RB;
  const int f = blockIdx.y;                         // position / problem b (or probe mode m)
  const bool FAR = a.farfield != 0;
  const int b = f, m = a.m, j = a.j;
  // input / output fields and stage configuration
  const float2* src = nullptr;
  float2* dst = nullptr;
  bool in_freq = true;     // S3/S4 from global (else natural spatial from global)
  int out = 1;             // 1: S1/S2 to global (x-transformed), 2: natural to global, 0: none
  int si = +1, so = -1;    // signs of the inverse-side (in) and forward (out) transforms
  const size_t fo = ((size_t)b * a.M + m) * NN;
  if (MODE == R_FWD) {
    src = (!FAR && j == 0) ? a.probe + (size_t)m * NN : a.FA + fo;
    in_freq = !((!FAR) && j == 0);
    dst = a.FA + fo;
    so = (FAR && j == a.L - 1) ? +1 : -1;
  } else if (MODE == R_RC_FIRST) {
    src = a.ckpt + (((size_t)b * a.M + m) * a.ncp + a.s) * NN;
    in_freq = false;
    dst = a.FR + fo;
  } else if (MODE == R_RC) {
    src = a.FR + fo;
    dst = a.FR + fo;
    out = (j < a.j1) ? 1 : 0;
  } else if (MODE == R_ADJ) {
    src = a.FA + fo;
    dst = a.FA + fo;
    si = (FAR && j == a.L - 1) ? -1 : +1;
    out = (!FAR && j == 0) ? 0 : 1;
  } else if (MODE == R_NEAR_DET || MODE == R_NEAR_SEED || MODE == R_NEAR_DSEED || MODE == R_NEAR_DSEED_P) {
    const size_t fd = (((size_t)b * (a.nd + 1) + a.d) * a.M + m) * NN;
    src = a.far + fd;
    dst = a.far + fd;
    in_freq = (MODE != R_NEAR_SEED);
    out = (MODE == R_NEAR_DET) ? 2 : 1;
  } else if (MODE == R_PHAT) {
    src = a.probe + (size_t)f * NN;
    dst = a.tmp + (size_t)f * NN;
    in_freq = false;
  } else if (MODE == R_PG_OUT) {
    src = a.tmp + (size_t)f * NN;
    out = 0;
  }
  __syncthreads();

  // ---- stage IN: S3 from global (natural kx = t + N1 i)
  if (in_freq) {
    for (int tau = threadIdx.x; tau < RB * N1; tau += NT2) {
      const int t = tau % N1, r = tau / N1;
      const float2* row = src + (size_t)(r0 + r) * N;
      float2 v[N2];
#pragma unroll
      for (int i = 0; i < N2; ++i) v[i] = row[t + N1 * i];
      if (si < 0) { dft<N2, -1>(v); twiddle<-1>(v, tw, t); }
      else { dft<N2, +1>(v); twiddle<+1>(v, tw, t); }
#pragma unroll
      for (int k = 0; k < N2; ++k) A[idx(r, N2 * t + k)] = v[k];
    }
    __syncthreads();
  }
  // ---- stage MID: S4 -> natural x = N2 k + t -> op -> S1
  Kahan lacc;   // R_NEAR_DSEED: loss terms of this thread's pixels
  for (int tau = threadIdx.x; tau < RB * N2; tau += NT2) {
    const int t = tau % N2, r = tau / N2;
    const int y = r0 + r;
    float2 v[N1];
    if (in_freq) {
#pragma unroll
      for (int k = 0; k < N1; ++k) v[k] = A[idx(r, N2 * k + t)];
      if (si < 0) dft<N1, -1>(v);
      else dft<N1, +1>(v);
    } else {
#pragma unroll
      for (int k = 0; k < N1; ++k) v[k] = src[(size_t)y * N + N2 * k + t];
    }
    // spatial ops; x = N2 k + t
    if (MODE == R_FWD || MODE == R_RC_FIRST || MODE == R_RC) {
      int p0y = 0, p0x = 0, gz = FAR ? j : b * a.L + j;
      if (FAR) {
        p0y = patch_corner(a.pos[2 * b]);
        p0x = patch_corner(a.pos[2 * b + 1]);
      }
      const int gy = p0y + y;
      const bool row_in = gy >= 0 && gy < a.Ly;
      float2* ck = a.ckpt + ((size_t)b * a.M + m) * a.ncp * NN;
      float2* sg = a.seg + ((size_t)b * a.M + m) * a.cp * NN;
      // transmission loads in chunks ahead of the checkpoint / segment stores
      constexpr int CH = N1 >= 32 ? 8 : N1;
#pragma unroll
      for (int k0 = 0; k0 < N1; k0 += CH) {
        float2 Tv[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          const int gx = p0x + N2 * (k0 + c) + t;
          const bool inb = row_in && gx >= 0 && gx < a.Lx;
          Tv[c] = inb ? __ldg(a.T + ((size_t)gz * a.Ly + gy) * a.Lx + gx) : make_float2(1.f, 0.f);
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          const int k = k0 + c;
          const float2 T = Tv[c];
          const size_t px = (size_t)y * N + N2 * k + t;
          if (MODE == R_FWD) {
            if (a.adj) {
              if (j % a.cp == 0) ck[(size_t)(j / a.cp) * NN + px] = v[k];
              else if (j > (a.ncp - 1) * a.cp) sg[(size_t)(j - (a.ncp - 1) * a.cp) * NN + px] = v[k];
            }
            v[k] = cmul(v[k], T);
          } else if (MODE == R_RC_FIRST) {
            v[k] = cmul(v[k], T);
          } else if (MODE == R_RC) {
            sg[(size_t)(j - a.j0) * NN + px] = v[k];
            v[k] = cmul(v[k], T);
          }
        }
      }
    }
    if (MODE == R_ADJ) {
      int p0y = 0, p0x = 0, gz = FAR ? j : b * a.L + j;
      if (FAR) {
        p0y = patch_corner(a.pos[2 * b]);
        p0x = patch_corner(a.pos[2 * b + 1]);
      }
      const int gy = p0y + y;
      const bool row_in = gy >= 0 && gy < a.Ly;
      const float2* psrc = (j == a.j0) ? a.ckpt + (((size_t)b * a.M + m) * a.ncp + a.s) * NN
                                       : a.seg + (((size_t)b * a.M + m) * a.cp + (j - a.j0)) * NN;
      // chunks of CH pixels: all loads of a chunk (T, psi and, in place, the gradient values)
      // are issued before any of its stores, so they are in flight together
      constexpr int CH = N1 >= 32 ? 4 : 8;
#pragma unroll
      for (int k0 = 0; k0 < N1; k0 += CH) {
        float2 Tv[CH], pv[CH];
        float gdv[CH], gbv[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          const int x = N2 * (k0 + c) + t, gx = p0x + x;
          const bool inb = row_in && gx >= 0 && gx < a.Lx;
          const size_t o = ((size_t)gz * a.Ly + gy) * a.Lx + gx;
          Tv[c] = inb ? __ldg(a.T + o) : make_float2(1.f, 0.f);
          pv[c] = __ldg(psrc + (size_t)y * N + x);
          if (a.gdf) {
            gdv[c] = a.gdf[o];
            gbv[c] = a.gbf[o];
          }
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          const int k = k0 + c, x = N2 * k + t, gx = p0x + x;
          const bool inb = row_in && gx >= 0 && gx < a.Lx;
          const size_t o = ((size_t)gz * a.Ly + gy) * a.Lx + gx;
          const float2 pbar = cmulc(v[k], Tv[c]);
          const float2 z = cmulc(pbar, pv[c]);
          if (a.gdf) {
            // near field, one mode: this thread owns the voxel for the whole call
            a.gdf[o] = gdv[c] + a.kdz * z.y;
            a.gbf[o] = gbv[c] - a.kdz * z.x;
          } else if (a.gd && inb) {
            atomicAdd(a.gd + o, f32_to_f64(a.kdz * z.y));
            atomicAdd(a.gb + o, f32_to_f64(-a.kdz * z.x));
          }
          v[k] = pbar;
          if (!FAR && j == 0 && a.qacc) a.qacc[fo + (size_t)y * N + x] = pbar;
        }
      }
    } else if (MODE == R_NEAR_DET) {
      float* g = a.gI + ((size_t)b * a.nd + a.d) * NN;
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        const size_t px = (size_t)y * N + N2 * k + t;
        const float I = fmaf(v[k].x, v[k].x, v[k].y * v[k].y);
        g[px] = (m == 0) ? I : g[px] + I;
      }
    } else if (MODE == R_NEAR_SEED) {
      const float* g = a.gI + ((size_t)b * a.nd + a.d) * NN;
#pragma unroll
      for (int k = 0; k < N1; ++k) v[k] = cscale(v[k], 2.0f * g[(size_t)y * N + N2 * k + t]);
    } else if (MODE == R_NEAR_DSEED || MODE == R_NEAR_DSEED_P) {
      const size_t pb = ((size_t)b * a.nd + a.d) * NN + (size_t)y * N + t;
      const float sc = 2.0f * (float)a.inv_npix;
      float im[N1];   // measured intensities first (read-only), then the I_out stores
#pragma unroll
      for (int k = 0; k < N1; ++k) im[k] = __ldg(a.I_meas + pb + N2 * k);
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        const float I = fmaf(v[k].x, v[k].x, v[k].y * v[k].y);
        if (a.I_out) a.I_out[pb + N2 * k] = I;
        float dI;
        lacc.add(loss_term(MODE == R_NEAR_DSEED_P ? 1 : 0, I, im[k], a.eps, &dI));
        v[k] = cscale(v[k], sc * dI);
      }
    } else if (MODE == R_PG_OUT) {
      float2* g = a.g_probe + (size_t)f * NN;
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        const size_t px = (size_t)y * N + N2 * k + t;
        g[px] = cadd(g[px], v[k]);
      }
    }
    if (out == 1) {
      if (so < 0) { dft<N1, -1>(v); twiddle<-1>(v, tw, t); }
      else { dft<N1, +1>(v); twiddle<+1>(v, tw, t); }
#pragma unroll
      for (int k = 0; k < N1; ++k) A[idx(r, N2 * k + t)] = v[k];
    } else if (out == 2) {
#pragma unroll
      for (int k = 0; k < N1; ++k) dst[(size_t)y * N + N2 * k + t] = v[k];
    }
  }
  if (MODE == R_NEAR_DSEED || MODE == R_NEAR_DSEED_P) {
    const double ls = block_sum2(lacc.value(), red);
    if (threadIdx.x == 0) a.lossp[((size_t)b * a.nd + a.d) * gridDim.x + blockIdx.x] = ls;
  }
  if (out != 1) return;
  __syncthreads();
  // ---- stage OUT: S2 to global (natural kx = t + N1 i)
  for (int tau = threadIdx.x; tau < RB * N1; tau += NT2) {
    const int t = tau % N1, r = tau / N1;
    float2 v[N2];
#pragma unroll
    for (int i = 0; i < N2; ++i) v[i] = A[idx(r, N2 * t + i)];
    if (so < 0) dft<N2, -1>(v);
    else dft<N2, +1>(v);
    float2* row = dst + (size_t)(r0 + r) * N;
#pragma unroll
    for (int i = 0; i < N2; ++i) row[t + N1 * i] = v[i];
  }
}

// ============================================================================ column kernel
template <int N, int MODE>
__global__ void __launch_bounds__(NT2, col_minb<N, MODE>()) k_col(const __grid_constant__ TPArgs a) {
  constexpr int N1 = Geo2<N>::N1, N2 = Geo2<N>::N2, CW = Geo2<N>::CW;
  constexpr size_t NN = (size_t)N * N;
  constexpr int BOXR = N < 256 ? N : 256;   // rows per TMA box
  extern __shared__ __align__(128) float2 sm[];
  float2* C = sm;
  float2* tw = C + N * CW;
  float2* ry = tw + N;
  float2* hy = ry + N;                // hy (far: propagator / near: detector factor of distance d)
  double* red = reinterpret_cast<double*>(hy + N);
  uint64_t* bar = reinterpret_cast<uint64_t*>(red + 64);
  const bool tma = a.tma != 0 && (smem_u32(C) & 127u) == 0;
  uint32_t phase = 0;
  if (tma && threadIdx.x == 0) mbar_init(bar);
  const int p0 = blockIdx.x * CW;
  const int f = blockIdx.y;
  const bool FAR = a.farfield != 0;
  const int b = f, m = a.m;
  const size_t fo = ((size_t)b * a.M + m) * NN;
  // propagator factors of this launch's gap (variable spacing) or the uniform ones
  const int gap = (MODE == C_PROP_ADJ) ? a.j - 1 : a.j;
  const float2* hysrc = (a.hyj && (MODE == C_PROP || MODE == C_PROP_ADJ)) ? a.hyj + (size_t)gap * N : a.hy;
  const float2* hxsrc = (a.hxj && (MODE == C_PROP || MODE == C_PROP_ADJ)) ? a.hxj + (size_t)gap * N : a.hx;
  for (int i = threadIdx.x; i < N; i += NT2) {
    tw[i] = a.tw[i];
    hy[i] = hysrc[i];
  }
  double dry = 0.0, drx = 0.0;
  if (FAR && (MODE == C_PSI0 || MODE == C_Q)) {
    const double py = a.pos[2 * b], px = a.pos[2 * b + 1];
    dry = py - floor(py + 0.5);
    drx = px - floor(px + 0.5);
    for (int i = threadIdx.x; i < N; i += NT2) ry[i] = shift_ramp((float)dry, i, N);
  }
  __syncthreads();

  // tensor map and first row of the field at src (a whole number of rows into FA, FR, far or tmp)
  auto tma_source = [&](const float2* src, int* which, int* row0) -> bool {
    const float2* bases[4] = {a.FA, a.FR, a.far, a.tmp};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (!bases[k] || src < bases[k]) continue;
      const size_t off = (size_t)(src - bases[k]);
      if (off >= (size_t)a.tm_rows[k] * N) continue;
      if (off % N) return false;
      *which = k;
      *row0 = (int)(off / N);
      return true;
    }
    return false;
  };
  // S1 of the column tile at src -> smem.  Returns false (for every thread of the CTA) when the
  // tile copy did not complete in time; the caller then leaves the kernel.
  auto stage_in = [&](const float2* src, int sgn) -> bool {
    int which = 0, row0 = 0;
    if (tma && tma_source(src, &which, &row0)) {
      // every earlier access of C is ordered before the asynchronous writes
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (threadIdx.x == 0) {
        mbar_expect_tx(bar, (uint32_t)(N * CW * sizeof(float2)));
#pragma unroll
        for (int yb = 0; yb < N / BOXR; ++yb) tma_load_2d(C + yb * BOXR * CW, &a.tm[which], p0, row0 + yb * BOXR, bar);
      }
      const bool ok = __syncthreads_and(mbar_wait_bounded(bar, phase, a.wait_tma));
      phase ^= 1u;
      if (!ok) {
        if (threadIdx.x == 0) set_status(a.status, STATUS_WAIT_TIMEOUT);
        mbar_wait_bounded(bar, phase ^ 1u);   // the copies still in flight land in this CTA's smem
        return false;
      }
      // in place: task (c, t) reads and writes the slots of rows N2 i + t of column c
      for (int tau = threadIdx.x; tau < CW * N2; tau += NT2) {
        const int c = tau % CW, t = tau / CW;
        float2 v[N1];
#pragma unroll
        for (int i = 0; i < N1; ++i) v[i] = C[(N2 * i + t) * CW + c];
        if (sgn < 0) { dft<N1, -1>(v); twiddle<-1>(v, tw, t); }
        else { dft<N1, +1>(v); twiddle<+1>(v, tw, t); }
#pragma unroll
        for (int k = 0; k < N1; ++k) C[(N2 * k + t) * CW + c] = v[k];
      }
      return true;
    }
    for (int tau = threadIdx.x; tau < CW * N2; tau += NT2) {
      const int c = tau % CW, t = tau / CW;
      float2 v[N1];
#pragma unroll
      for (int i = 0; i < N1; ++i) v[i] = src[(size_t)(N2 * i + t) * N + p0 + c];
      if (sgn < 0) { dft<N1, -1>(v); twiddle<-1>(v, tw, t); }
      else { dft<N1, +1>(v); twiddle<+1>(v, tw, t); }
#pragma unroll
      for (int k = 0; k < N1; ++k) C[(N2 * k + t) * CW + c] = v[k];
    }
    return true;
  };
  // S4 from smem -> global column tile (natural y)
  auto stage_out = [&](float2* dst, int sgn) {
    for (int tau = threadIdx.x; tau < CW * N2; tau += NT2) {
      const int c = tau % CW, t = tau / CW;
      float2 v[N1];
#pragma unroll
      for (int i = 0; i < N1; ++i) v[i] = C[(N2 * i + t) * CW + c];
      if (sgn < 0) dft<N1, -1>(v);
      else dft<N1, +1>(v);
#pragma unroll
      for (int k = 0; k < N1; ++k) dst[(size_t)(N2 * k + t) * N + p0 + c] = v[k];
    }
  };
  // S3 of registers -> smem
  auto s3_store = [&](float2 (&v)[N2], int c, int t, int sgn) {
    if (sgn < 0) { dft<N2, -1>(v); twiddle<-1>(v, tw, t); }
    else { dft<N2, +1>(v); twiddle<+1>(v, tw, t); }
#pragma unroll
    for (int k = 0; k < N2; ++k) C[(N2 * t + k) * CW + c] = v[k];
  };
  auto s2_load = [&](float2 (&v)[N2], int c, int t, int sgn) {
#pragma unroll
    for (int i = 0; i < N2; ++i) v[i] = C[(N2 * t + i) * CW + c];
    if (sgn < 0) dft<N2, -1>(v);
    else dft<N2, +1>(v);
  };

  if (MODE == C_PROP || MODE == C_PROP_ADJ) {
    float2* F = (a.buf == 1 ? a.FR : a.FA) + fo;
    // slice-gap gradient: keep F[psi_{gap+1}] / N^2 (forward / recompute), or accumulate
    // -pi sum |f|^2 Im(conj(F[psibar]) F[psi]) against the kept spectrum (adjoint)
    float2* so = (MODE == C_PROP && a.spec_out)
                     ? a.spec_out + (((size_t)b * a.M + m) * a.spo_n + a.spo_slot) * NN : nullptr;
    const float2* si = (MODE == C_PROP_ADJ && a.spec_in)
                           ? a.spec_in + (((size_t)b * a.M + m) * a.spi_n + a.spi_slot) * NN : nullptr;
    if (!stage_in(F, -1)) return;
    __syncthreads();
    float gs = 0.f;
    for (int tau = threadIdx.x; tau < CW * N1; tau += NT2) {
      const int c = tau % CW, t = tau / CW, kx = p0 + c;
      float2 v[N2];
      s2_load(v, c, t, -1);
      const float2 hx = hxsrc[kx];
      const float fx = freqf(kx, N);
#pragma unroll
      for (int i = 0; i < N2; ++i) {
        const int ky = t + N1 * i;
        const float2 h = cmul(hy[ky], hx);
        if (MODE == C_PROP) {
          v[i] = cmul(v[i], h);
          if (so) so[(size_t)ky * N + kx] = v[i];
        } else {
          if (si) {
            const float fy = freqf(ky, N);
            gs += (fy * fy + fx * fx) * cmulc(si[(size_t)ky * N + kx], v[i]).y;
          }
          v[i] = cmulc(v[i], h);
        }
      }
      s3_store(v, c, t, +1);
    }
    __syncthreads();
    stage_out(F, +1);
    if (si && a.gapp) {
      const double g = block_sum2(f32_to_f64(gs), red);
      if (threadIdx.x == 0) {
        double* gp = a.gapp + (((size_t)b * (a.L - 1) + gap) * gridDim.x + blockIdx.x);
        const double val = -3.14159265358979323846 * g;
        *gp = (m == 0) ? val : *gp + val;
      }
    }
  } else if (MODE == C_PSI0 || MODE == C_SEED || MODE == C_PG) {
    // Fourier-space input from op, inverse y-transform to global
    for (int tau = threadIdx.x; tau < CW * N1; tau += NT2) {
      const int c = tau % CW, t = tau / CW;
      const int kx = p0 + c;
      float2 v[N2];
      if (MODE == C_PSI0) {
        const float2* ph = a.phat + (size_t)m * NN;
        const float2 rx = cscale(shift_ramp((float)drx, kx, N), 1.0f / (float)NN);
#pragma unroll
        for (int i = 0; i < N2; ++i) {
          const int ky = t + N1 * i;
          v[i] = cmul(cmul(ph[(size_t)ky * N + kx], ry[ky]), rx);
        }
      } else if (MODE == C_SEED) {
        const float2* fm = a.far + fo;
        const float* g = a.gI + (size_t)b * NN;
        const float sc = 2.0f / (float)N;
#pragma unroll
        for (int i = 0; i < N2; ++i) {
          const size_t p = (size_t)(t + N1 * i) * N + kx;
          v[i] = cscale(fm[p], sc * g[p]);
        }
      } else {   // C_PG: qsum / N^2
        const float2* q = a.qsum + (size_t)f * NN;
#pragma unroll
        for (int i = 0; i < N2; ++i) v[i] = cscale(q[(size_t)(t + N1 * i) * N + kx], 1.0f / (float)NN);
      }
      s3_store(v, c, t, MODE == C_SEED ? -1 : +1);
    }
    __syncthreads();
    float2* dst = (MODE == C_PG) ? a.tmp + (size_t)f * NN : a.FA + fo;
    stage_out(dst, MODE == C_SEED ? -1 : +1);
  } else if (MODE == C_FAR || MODE == C_Q || MODE == C_PHAT) {
    const int sg = (MODE == C_FAR) ? +1 : -1;
    const float2* F = (MODE == C_PHAT) ? a.tmp + (size_t)f * NN : a.FA + fo;
    if (!stage_in(F, sg)) return;
    __syncthreads();
    float ay = 0.f, ax = 0.f;
    for (int tau = threadIdx.x; tau < CW * N1; tau += NT2) {
      const int c = tau % CW, t = tau / CW;
      const int kx = p0 + c;
      float2 v[N2];
      s2_load(v, c, t, sg);
      if (MODE == C_FAR) {
        float2* fm = a.far + fo;
        float* g = a.gI + (size_t)b * NN;
        const float invN = 1.0f / (float)N;
#pragma unroll
        for (int i = 0; i < N2; ++i) {
          const size_t p = (size_t)(t + N1 * i) * N + kx;
          const float2 P = cscale(v[i], invN);
          fm[p] = P;
          const float I = fmaf(P.x, P.x, P.y * P.y);
          g[p] = (m == 0) ? I : g[p] + I;
        }
      } else if (MODE == C_PHAT) {
        float2* o = a.phat_w + (size_t)f * NN;
#pragma unroll
        for (int i = 0; i < N2; ++i) o[(size_t)(t + N1 * i) * N + kx] = v[i];
      } else {   // C_Q
        const float2* ph = a.phat + (size_t)m * NN;
        float2* q = a.qacc ? a.qacc + fo : nullptr;
        const float2 rx = shift_ramp((float)drx, kx, N);
        const float fx = freqf(kx, N);
#pragma unroll
        for (int i = 0; i < N2; ++i) {
          const int ky = t + N1 * i;
          const size_t p = (size_t)ky * N + kx;
          const float2 r = cmul(ry[ky], rx);
          const float2 base = cmul(cconj(v[i]), cmul(ph[p], r));
          ay += freqf(ky, N) * base.y;
          ax += fx * base.y;
          if (q) q[p] = cmulc(v[i], r);
        }
      }
    }
    if (MODE == C_Q && a.posp) {
      double sm3[3];
      block_sum3(ay, ax, 0.f, red, sm3);
      const double sy = sm3[0], sx = sm3[1];
      if (threadIdx.x == 0) {
        double* pp = a.posp + ((size_t)b * gridDim.x + blockIdx.x) * 3;
        pp[0] = (m == 0) ? sy : pp[0] + sy;
        pp[1] = (m == 0) ? sx : pp[1] + sx;
        pp[2] = 0.0;
      }
    }
  } else if (MODE == C_FAR_SEED || MODE == C_FAR_SEED_P) {
    // Psi = (1/N) DFT_+[phi_{L-1}] -> I, loss term, dL/dI -> phibar_{L-1} = (1/N) DFT_-[2 dL/dI Psi]
    if (!stage_in(a.FA + fo, +1)) return;
    __syncthreads();
    const float invN = 1.0f / (float)N, sc = 2.0f * invN * (float)a.inv_npix;
    const size_t pb = (size_t)b * NN;
    Kahan lacc;
    for (int tau = threadIdx.x; tau < CW * N1; tau += NT2) {
      const int c = tau % CW, t = tau / CW, kx = p0 + c;
      float im[N2];   // measured intensities first (read-only), then the I_out stores
#pragma unroll
      for (int i = 0; i < N2; ++i) im[i] = __ldg(a.I_meas + pb + (size_t)(t + N1 * i) * N + kx);
      float2 v[N2];
      s2_load(v, c, t, +1);
#pragma unroll
      for (int i = 0; i < N2; ++i) {
        const size_t px = pb + (size_t)(t + N1 * i) * N + kx;
        const float2 P = cscale(v[i], invN);
        const float I = fmaf(P.x, P.x, P.y * P.y);
        if (a.I_out) a.I_out[px] = I;
        float dI;
        lacc.add(loss_term(MODE == C_FAR_SEED_P ? 1 : 0, I, im[i], a.eps, &dI));
        v[i] = cscale(P, sc * dI);
      }
      s3_store(v, c, t, -1);
    }
    __syncthreads();
    stage_out(a.FA + fo, -1);
    const double ls = block_sum2(lacc.value(), red);
    if (threadIdx.x == 0) a.lossp[(size_t)b * gridDim.x + blockIdx.x] = ls;
  } else if (MODE == C_NEAR_PHI) {
    // Phi = DFT_-[phi] (stored for the shift gradients); then for each distance
    // Psi_d = IDFT_-{Phi G_d}: y-inverse here, x-inverse in the row kernel.  Each thread reads
    // back the Phi values it stored itself (no barrier needed; they are L2-resident)
    if (!stage_in(a.FA + fo, -1)) return;
    __syncthreads();
    float2* Phi = a.far + (((size_t)b * (a.nd + 1) + a.nd) * a.M + m) * NN;
    for (int tau = threadIdx.x; tau < CW * N1; tau += NT2) {
      const int c = tau % CW, t = tau / CW;
      float2 v[N2];
      s2_load(v, c, t, -1);
#pragma unroll
      for (int i = 0; i < N2; ++i) Phi[(size_t)(t + N1 * i) * N + p0 + c] = v[i];
    }
    for (int d = 0; d < a.nd; ++d) {
      const float sy = a.pos[((size_t)b * a.nd + d) * 2], sx = a.pos[((size_t)b * a.nd + d) * 2 + 1];
      __syncthreads();   // every S2 read (d = 0) / S4 read (d > 0) of the tile is done
      for (int i = threadIdx.x; i < N; i += NT2) ry[i] = cmul(shift_ramp(sy, i, N), a.hd[(size_t)d * N + i]);
      __syncthreads();
      for (int tau = threadIdx.x; tau < CW * N1; tau += NT2) {
        const int c = tau % CW, t = tau / CW, kx = p0 + c;
        const float2 gx = cscale(cmul(shift_ramp(sx, kx, N), a.hd[(size_t)d * N + kx]), 1.0f / (float)NN);
        float2 v[N2];
#pragma unroll
        for (int i = 0; i < N2; ++i) v[i] = cmul(cmul(Phi[(size_t)(t + N1 * i) * N + kx], ry[t + N1 * i]), gx);
        s3_store(v, c, t, +1);
      }
      __syncthreads();
      stage_out(a.far + (((size_t)b * (a.nd + 1) + d) * a.M + m) * NN, +1);
    }
  } else if (MODE == C_NEAR_Q) {
    // Q_d = DFT_-[seed_d]; shift-gradient partials; phibar = IDFT_-{sum_d conj(G_d) Q_d}.  The sum
    // over distances is kept in this CTA's own columns of FA (consumed by C_NEAR_PHI, rewritten by
    // the stage_out below): each thread adds into the slots it alone owns, L2-resident
    const float2* Phi = a.far + (((size_t)b * (a.nd + 1) + a.nd) * a.M + m) * NN;
    float2* acc = a.FA + fo;
    for (int d = 0; d < a.nd; ++d) {
      const float sy = a.pos[((size_t)b * a.nd + d) * 2], sx = a.pos[((size_t)b * a.nd + d) * 2 + 1];
      __syncthreads();
      if (!stage_in(a.far + (((size_t)b * (a.nd + 1) + d) * a.M + m) * NN, -1)) return;
      for (int i = threadIdx.x; i < N; i += NT2) ry[i] = cmul(shift_ramp(sy, i, N), a.hd[(size_t)d * N + i]);
      __syncthreads();
      float ay = 0.f, ax = 0.f, an = 0.f;
      for (int tau = threadIdx.x; tau < CW * N1; tau += NT2) {
        const int c = tau % CW, t = tau / CW, kx = p0 + c;
        const float2 gx = cmul(shift_ramp(sx, kx, N), a.hd[(size_t)d * N + kx]);
        const float fx = freqf(kx, N);
        float2 v[N2];
        s2_load(v, c, t, -1);
        // Phi and the running sum in chunks, loaded ahead of the chunk's stores
        constexpr int CH = 8;
#pragma unroll
        for (int i0 = 0; i0 < N2; i0 += CH) {
          float2 ph[CH], ac[CH];
#pragma unroll
          for (int e = 0; e < CH; ++e) {
            const size_t p = (size_t)(t + N1 * (i0 + e)) * N + kx;
            ph[e] = __ldg(Phi + p);
            ac[e] = (d == 0) ? make_float2(0.f, 0.f) : acc[p];
          }
#pragma unroll
          for (int e = 0; e < CH; ++e) {
            const int i = i0 + e, ky = t + N1 * i;
            const float fy = freqf(ky, N);
            const float2 G = cmul(ry[ky], gx);
            const float2 base = cmul(cconj(v[i]), cmul(ph[e], G));
            ay += fy * base.y;
            ax += fx * base.y;
            an += (fy * fy + fx * fx) * base.y;
            acc[(size_t)ky * N + kx] = cadd(ac[e], cmulc(v[i], G));
          }
        }
      }
      if (a.posp) {
        double sm3[3];
        block_sum3(ay, ax, an, red, sm3);
        const double s_y = sm3[0], s_x = sm3[1], s_n = sm3[2];
        if (threadIdx.x == 0) {
          double* pp = a.posp + (((size_t)b * a.nd + d) * gridDim.x + blockIdx.x) * 3;
          pp[0] = (m == 0) ? s_y : pp[0] + s_y;
          pp[1] = (m == 0) ? s_x : pp[1] + s_x;
          pp[2] = (m == 0) ? s_n : pp[2] + s_n;
        }
      }
    }
    __syncthreads();
    for (int tau = threadIdx.x; tau < CW * N1; tau += NT2) {
      const int c = tau % CW, t = tau / CW, kx = p0 + c;
      float2 v[N2];
#pragma unroll
      for (int i = 0; i < N2; ++i) v[i] = cscale(acc[(size_t)(t + N1 * i) * N + kx], 1.0f / (float)NN);
      s3_store(v, c, t, +1);
    }
    __syncthreads();
    stage_out(a.FA + fo, +1);
  }
}

// ============================================================================ loss, final reductions
constexpr int LOSS_PX = 1024;   // pixels per loss CTA (256 threads x 4)

__global__ void __launch_bounds__(256) k_loss2(const TPArgs a) {
  __shared__ double red[8];
  const size_t NN = (size_t)a.N * a.N;
  const size_t base = (size_t)blockIdx.y * NN;
  Kahan acc;
  for (int e = 0; e < 4; ++e) {
    const size_t p = base + (size_t)blockIdx.x * LOSS_PX + e * 256 + threadIdx.x;
    const float I = a.gI[p];
    if (a.I_out) a.I_out[p] = I;
    if (!a.I_meas) continue;
    float dI;
    acc.add(loss_term(a.loss, I, a.I_meas[p], a.eps, &dI));
    a.gI[p] = dI * (float)a.inv_npix;
  }
  const double s = block_sum2(acc.value(), red);
  if (threadIdx.x == 0) a.lossp[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// loss: all threads over the partials, fixed split and order; shift / Fresnel-number gradients: one
// warp per (problem, distance), lanes over the column-CTA partials, fixed shuffle tree
__global__ void __launch_bounds__(1024) k_final2(const TPArgs a, int nloss, int ncolblk) {
  __shared__ double red[32];
  if (a.loss_out) {
    const int chunk = (nloss + blockDim.x - 1) / blockDim.x;
    double acc = 0.0;
    for (int i = threadIdx.x * chunk; i < min(nloss, (int)(threadIdx.x + 1) * chunk); ++i) acc += a.lossp[i];
    const double s = block_sum2(acc, red);
    if (threadIdx.x == 0) *a.loss_out = s * a.inv_npix;
  }
  if (a.posp && (a.gpos || a.gposd || a.gnf)) {
    const double pi = 3.14159265358979323846, NN = (double)a.N * a.N, sc = 2.0 * pi / NN;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int q = w; q < a.B * a.nd; q += nw) {
      double sy = 0.0, sx = 0.0, sn = 0.0;
      for (int k = l; k < ncolblk; k += 32) {
        const double* pp = a.posp + ((size_t)q * ncolblk + k) * 3;
        sy += pp[0];
        sx += pp[1];
        sn += pp[2];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sn += __shfl_xor_sync(0xffffffffu, sn, o);
      }
      if (l == 0) {
        if (a.gpos) {
          a.gpos[2 * q] = (float)(sc * sy);
          a.gpos[2 * q + 1] = (float)(sc * sx);
        }
        if (a.gposd) {   // far field (one distance): q is the position
          a.gposd[2 * q] = sc * sy;
          a.gposd[2 * q + 1] = sc * sx;
        }
        if (a.gnf) {
          const double nf = a.nf[q % a.nd];
          a.gnf[q] = (float)(pi * sn / (nf * nf * NN));
        }
      }
    }
  }
}

__global__ void k_add2(float2* __restrict__ g, const float2* __restrict__ q, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    g[i] = cadd(g[i], q[i]);
}

// ============================================================================ launch sequence
template <int N, int MODE>
static void row(const TPArgs& a, int gy, cudaStream_t s) {
  (k_row<N, MODE><<<dim3(N / Geo2<N>::RB, gy), NT2, row_smem_bytes<N>(), s>>>(a), note_launch());
}
template <int N, int MODE>
static void col(const TPArgs& a, int gy, cudaStream_t s) {
  (k_col<N, MODE><<<dim3(N / Geo2<N>::CW, gy), NT2, col_smem_bytes<N>(), s>>>(a), note_launch());
}

template <int N, class F>
static cudaError_t set_attr(F* k, int bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <int N>
static cudaError_t prepare_t2() {
  cudaError_t e = cudaSuccess;
  const int rb = row_smem_bytes<N>(), cb = col_smem_bytes<N>();
#define ROWA(M_) if (e == cudaSuccess) e = set_attr<N>(k_row<N, M_>, rb);
#define COLA(M_) if (e == cudaSuccess) e = set_attr<N>(k_col<N, M_>, cb);
  ROWA(R_FWD) ROWA(R_RC_FIRST) ROWA(R_RC) ROWA(R_ADJ) ROWA(R_NEAR_DET) ROWA(R_NEAR_SEED) ROWA(R_PHAT) ROWA(R_PG_OUT) ROWA(R_NEAR_DSEED) ROWA(R_NEAR_DSEED_P)
  COLA(C_PROP) COLA(C_PROP_ADJ) COLA(C_PSI0) COLA(C_FAR) COLA(C_SEED) COLA(C_Q) COLA(C_PHAT) COLA(C_PG)
  COLA(C_NEAR_PHI) COLA(C_NEAR_Q) COLA(C_FAR_SEED) COLA(C_FAR_SEED_P)
#undef ROWA
#undef COLA
  return e;
}


cudaError_t prepare_twopass(int N) {
  // idempotent; called by every entry point before it enqueues (never inside a stream capture)
  const int i = N == 256 ? 0 : N == 512 ? 1 : N == 1024 ? 2 : -1;
  if (i < 0) return cudaErrorInvalidValue;
  static std::atomic<bool> prepared[kMaxDevices][3] = {};
  const int dev = current_device();
  if (dev >= 0 && prepared[dev][i].load(std::memory_order_acquire)) return cudaSuccess;
  cudaError_t e = N == 256 ? prepare_t2<256>() : N == 512 ? prepare_t2<512>() : prepare_t2<1024>();
  if (e == cudaSuccess && dev >= 0) prepared[dev][i].store(true, std::memory_order_release);
  return e;
}

// ADORYM_TMA_STAGING=0 builds the register-staged column loads only (for comparisons)
#ifndef ADORYM_TMA_STAGING
#define ADORYM_TMA_STAGING 1
#endif

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against the driver)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  // looked up once per process (thread-safe initialisation of a function-local static)
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
    return nullptr;
  }();
  return fn;
}

// 2-D map over `rows` rows of N complex64 (8-byte elements) at base, box CW x min(N, 256).  The
// TMA rules are checked here: base 16-byte aligned, row stride and box width multiples of 16
// bytes (every x coordinate the kernels use is a multiple of CW, i.e. of 16 bytes).
template <int N>
static bool encode_tile_map(CUtensorMap* m, const void* base, unsigned long long rows) {
  constexpr int CW = Geo2<N>::CW;
  static_assert((CW * sizeof(float2)) % 16 == 0 && (N * sizeof(float2)) % 16 == 0, "TMA alignment");
  auto fn = tensor_map_encoder();
  if (!fn || !base || rows == 0 || (reinterpret_cast<uintptr_t>(base) & 15u)) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)N * sizeof(float2)};
  const cuuint32_t box[2] = {(cuuint32_t)CW, (cuuint32_t)std::min(N, 256)};
  const cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_INT64, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int N>
static cudaError_t twopass_t(TPArgs a, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1, cudaEvent_t meas_ready,
                             const cudaEvent_t* meas_part, int n_meas_part) {
  const bool far = a.farfield != 0;
  const int B = a.B, M = a.M, L = a.L;
  const size_t NN = (size_t)N * N;
  {
    // tile maps of the column kernels' sources: FA, FR (adjoint only), far, tmp
    const void* bases[4] = {a.FA, a.FR, a.far, a.tmp};
    const unsigned long long rows[4] = {(unsigned long long)B * M * N, a.FR ? (unsigned long long)B * M * N : 0ull,
                                        (unsigned long long)B * (far ? 1 : a.nd + 1) * M * N,
                                        (unsigned long long)M * N};
    bool ok = a.status != nullptr;
    for (int k = 0; k < 4 && ok; ++k) {
      a.tm_rows[k] = bases[k] ? rows[k] : 0ull;
      if (bases[k]) ok = encode_tile_map<N>(&a.tm[k], bases[k], rows[k]);
    }
    a.tma = (ok && ADORYM_TMA_STAGING) ? 1 : 0;
  }
  // slice-gap gradient: spectra of checkpoint slices [B][M][ncp] and of segment slices [B][M][cp]
  float2* spck = a.spec_out;
  float2* spsg = const_cast<float2*>(a.spec_in);
  const bool want_gap = a.adj && a.gapp && spck && spsg;
  const int j0_last = (a.ncp - 1) * a.cp;
  a.spec_out = nullptr;
  a.spec_in = nullptr;
  auto out_slot = [&](float2* base, int n, int slot) {
    a.spec_out = want_gap ? base : nullptr;
    a.spo_n = n;
    a.spo_slot = slot;
  };
  const int ncol = N / Geo2<N>::CW;
  // one probe mode with measured data: loss and adjoint seed fused into the detector pass
  const bool fuse = a.adj && M == 1 && a.I_meas != nullptr;
  const int nloss = !fuse ? (int)(B * a.nd * (NN / LOSS_PX)) : far ? B * ncol : B * a.nd * (N / Geo2<N>::RB);
  // the detector passes (and the separate loss pass) are the first readers of the measured
  // intensities: wait for their copy there, not before the forward passes
  cudaError_t werr = cudaSuccess;
  auto wait_meas = [&]() {
    if (!meas_ready) return;
    const cudaError_t e = cudaStreamWaitEvent(s, meas_ready, 0);
    if (e != cudaSuccess && werr == cudaSuccess) werr = e;
    meas_ready = nullptr;
  };
  if (ev0) cudaEventRecord(ev0, s);
  if (far) {
    row<N, R_PHAT>(a, M, s);
    col<N, C_PHAT>(a, M, s);
  }
  // ---------------- forward
  for (int m = 0; m < M; ++m) {
    a.m = m;
    if (far) col<N, C_PSI0>(a, B, s);
    for (int j = 0; j < L; ++j) {
      a.j = j;
      row<N, R_FWD>(a, B, s);
      if (j < L - 1) {
        a.buf = 0;
        const int jn = j + 1;
        if (jn % a.cp == 0) out_slot(spck, a.ncp, jn / a.cp);
        else if (jn > j0_last) out_slot(spsg, a.cp, jn - j0_last);
        else out_slot(nullptr, 1, 0);
        col<N, C_PROP>(a, B, s);
        a.spec_out = nullptr;
      } else if (far) {
        wait_meas();
        if (fuse && a.loss == 1) col<N, C_FAR_SEED_P>(a, B, s);
        else if (fuse) col<N, C_FAR_SEED>(a, B, s);
        else col<N, C_FAR>(a, B, s);
      } else {
        col<N, C_NEAR_PHI>(a, B, s);
        const bool parts = meas_ready && meas_part && n_meas_part == a.nd;
        if (!parts) wait_meas();
        for (int d = 0; d < a.nd; ++d) {
          a.d = d;
          if (parts) {   // this distance's intensities only; the later ones are still arriving
            const cudaError_t e = cudaStreamWaitEvent(s, meas_part[d], 0);
            if (e != cudaSuccess && werr == cudaSuccess) werr = e;
          }
          if (fuse && a.loss == 1) row<N, R_NEAR_DSEED_P>(a, B, s);
          else if (fuse) row<N, R_NEAR_DSEED>(a, B, s);
          else row<N, R_NEAR_DET>(a, B, s);
        }
      }
    }
  }
  wait_meas();   // (no-op when a detector pass already waited)
  if (!fuse) (k_loss2<<<dim3((unsigned)(NN / LOSS_PX), B * a.nd), 256, 0, s>>>(a), note_launch());
  if (a.adj) {
    // ---------------- adjoint
    for (int m = 0; m < M; ++m) {
      a.m = m;
      if (far) {
        if (!fuse) col<N, C_SEED>(a, B, s);
      } else {
        if (!fuse) {
          for (int d = 0; d < a.nd; ++d) {
            a.d = d;
            row<N, R_NEAR_SEED>(a, B, s);
          }
        }
        col<N, C_NEAR_Q>(a, B, s);
      }
      for (int sg = a.ncp - 1; sg >= 0; --sg) {
        const int j0 = sg * a.cp, j1 = min(j0 + a.cp, L) - 1;
        a.s = sg;
        a.j0 = j0;
        a.j1 = j1;
        if (sg != a.ncp - 1 && j1 > j0) {
          a.j = j0;
          row<N, R_RC_FIRST>(a, B, s);
          for (int j = j0 + 1; j <= j1; ++j) {
            a.buf = 1;
            a.j = j - 1;                                  // gap j-1 -> j
            out_slot(spsg, a.cp, j - j0);
            col<N, C_PROP>(a, B, s);
            a.spec_out = nullptr;
            a.j = j;
            row<N, R_RC>(a, B, s);
          }
        }
        for (int j = j1; j >= j0; --j) {
          a.j = j;
          row<N, R_ADJ>(a, B, s);
          if (j > 0) {
            a.buf = 0;
            if (want_gap) {
              a.spec_in = (j == j0) ? spck : spsg;
              a.spi_n = (j == j0) ? a.ncp : a.cp;
              a.spi_slot = (j == j0) ? sg : j - j0;
            }
            col<N, C_PROP_ADJ>(a, B, s);
            a.spec_in = nullptr;
          } else if (far) {
            col<N, C_Q>(a, B, s);
          }
        }
      }
    }
  }
  if (ev1) cudaEventRecord(ev1, s);
  if (a.adj) {
    (k_final2<<<1, 1024, 0, s>>>(a, nloss, ncol), note_launch());
    if (want_gap && a.ggap) launch_gap_final(a.gapp, B, L - 1, ncol, a.ggap, s);
    if (a.g_probe) {
      const size_t MNN = (size_t)M * NN;
      // per-element FP64 sum over the batch (deterministic), then back to real space
      launch_qsum(a.qacc, a.qsum, B, MNN, s);
      if (far) {
        col<N, C_PG>(a, M, s);
        row<N, R_PG_OUT>(a, M, s);
      } else {
        (k_add2<<<1024, 256, 0, s>>>(a.g_probe, a.qsum, MNN), note_launch());
      }
    }
  }
  const cudaError_t e = cudaGetLastError();
  return e != cudaSuccess ? e : werr;
}

cudaError_t launch_twopass(TPArgs a, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1, cudaEvent_t meas_ready,
                           const cudaEvent_t* meas_part, int n_meas_part) {
  switch (a.N) {
    case 256: return twopass_t<256>(a, s, ev0, ev1, meas_ready, meas_part, n_meas_part);
    case 512: return twopass_t<512>(a, s, ev0, ev1, meas_ready, meas_part, n_meas_part);
    case 1024: return twopass_t<1024>(a, s, ev0, ev1, meas_ready, meas_part, n_meas_part);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace adorym
