// Launchers of the fused kernel without per-gap propagators, and the per-call probe kernels
// around it (probe DFT, probe-gradient reduction, slice-gap gradient reduction).
#include "k_path.cuh"

namespace adorym {

// ---------------------------------------------------------------------------- probe DFT
template <int N>
__global__ void __launch_bounds__(Geo<N>::NT) k_probe_hat(const float2* __restrict__ probe, float2* __restrict__ phat,
                                                        const float2* __restrict__ twg) {
  using F = Field<N>;
  constexpr int N1 = F::N1, N2 = F::N2;
  extern __shared__ float2 sm[];
  float2* A = sm;
  float2* tw = A + N * F::LD;
  F::fill_twiddles(tw, twg);
  __syncthreads();
  const float2* p = probe + (size_t)blockIdx.x * N * N;
  float2* o = phat + (size_t)blockIdx.x * N * N;
  using V1 = float2[N1];
  using V2 = float2[N2];
  pass_c14<N, 0, -1, false, true>(A, tw, NoPre(), [&](V1& v, V1&, V1&, int x, int t) {
#pragma unroll
    for (int k = 0; k < N1; ++k) v[k] = p[(N2 * k + t) * N + x];
  });
  __syncthreads();
  pass_c23<N, false, -1>(A, tw);
  __syncthreads();
  pass_r14<N, true, -1>(A, tw);
  __syncthreads();
  pass_r23<N, -1, 0>(A, tw, [&](V2& v, int ky, int t) {
#pragma unroll
    for (int i = 0; i < N2; ++i) o[ky * N + t + N1 * i] = v[i];
  });
}

// ---------------------------------------------------------------------------- probe gradient
// qsum[m][p] = sum_b qacc[b][m][p] in FP64, fixed order
// Block of 256 threads = 32 consecutive elements x 8 batch chunks; each thread sums its chunk
// Kahan-compensated in FP32 (loads issued four at a time), then the 8 partials of an element are
// added in FP64 in chunk order (deterministic).
__global__ void __launch_bounds__(256) k_qsum(const float2* __restrict__ qacc, float2* __restrict__ qsum, int B,
                                              size_t MNN) {
  __shared__ double2 part[8][32];
  const int e = threadIdx.x & 31, c = threadIdx.x >> 5;
  const size_t i = (size_t)blockIdx.x * 32 + e;
  const int b0 = (B * c) / 8, b1 = (B * (c + 1)) / 8;
  Kahan sr, si;
  if (i < MNN) {
#pragma unroll 4
    for (int b = b0; b < b1; ++b) {
      const float2 v = __ldg(qacc + (size_t)b * MNN + i);
      sr.add(v.x);
      si.add(v.y);
    }
  }
  part[c][e] = make_double2(sr.value(), si.value());
  __syncthreads();
  if (c == 0 && i < MNN) {
    double r = 0.0, im = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      r += part[k][e].x;
      im += part[k][e].y;
    }
    qsum[i] = make_float2((float)r, (float)im);
  }
}

__global__ void k_gap_final(const double* __restrict__ gapp, int B, int ngap, int parts, float* __restrict__ g) {
  for (int j = threadIdx.x; j < ngap; j += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < B; ++b)
      for (int k = 0; k < parts; ++k) s += gapp[((size_t)b * ngap + j) * parts + k];
    g[j] = (float)s;
  }
}

// Per-angle position offset of ptychotomography (Sec. 2.3.2): one correction vector shifts every
// position of an angle, so its gradient is the sum of that batch's position gradients.  One warp:
// lane l adds positions l, l + 32, ... in FP64, then a fixed shuffle tree (deterministic).
__global__ void k_offset_sum(const double* __restrict__ gposd, int B, float* __restrict__ g_off) {
  double sy = 0.0, sx = 0.0;
  for (int b = threadIdx.x; b < B; b += 32) {
    sy += gposd[2 * (size_t)b];
    sx += gposd[2 * (size_t)b + 1];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sy += __shfl_xor_sync(0xffffffffu, sy, o);
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
  }
  if (threadIdx.x == 0) {
    g_off[0] = (float)sy;
    g_off[1] = (float)sx;
  }
}

cudaError_t launch_offset_sum(const double* gposd, int B, float* g_off, cudaStream_t s) {
  (k_offset_sum<<<1, 32, 0, s>>>(gposd, B, g_off), note_launch());
  return cudaGetLastError();
}

cudaError_t launch_gap_final(const double* gapp, int B, int ngap, int parts, float* g_gap, cudaStream_t s) {
  (k_gap_final<<<1, 256, 0, s>>>(gapp, B, ngap, parts, g_gap), note_launch());
  return cudaGetLastError();
}

cudaError_t launch_qsum(const float2* qacc, float2* qsum, int B, size_t MNN, cudaStream_t s) {
  (k_qsum<<<(unsigned)((MNN + 31) / 32), 256, 0, s>>>(qacc, qsum, B, MNN), note_launch());
  return cudaGetLastError();
}

// far field: g_probe[m] += IDFT_-{qsum[m]};  near field: g_probe[m] += qsum[m]
template <int N, int FAR>
__global__ void __launch_bounds__(Geo<N>::NT) k_probe_grad(const float2* __restrict__ qsum, float2* __restrict__ g,
                                                         const float2* __restrict__ twg, const double* __restrict__ lossp,
                                                         int B, double inv_npix, double* __restrict__ loss_out) {
  using F = Field<N>;
  constexpr int N1 = F::N1, N2 = F::N2, NT = F::NT;
  constexpr size_t NN = (size_t)N * N;
  extern __shared__ float2 sm[];
  float2* A = sm;
  float2* tw = A + N * F::LD;
  if (loss_out && blockIdx.x == 0 && threadIdx.x < 32) {
    // FP64 sum of the per-position partials in a fixed order: lane l adds positions l, l + 32, ...
    // in turn, then a fixed xor tree over the lanes (one warp keeps B / 32 loads in flight instead of
    // one thread walking all B partials)
    double s = 0.0;
    for (int b = (int)threadIdx.x; b < B; b += 32) s += lossp[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *loss_out = s * inv_npix;
  }
  if (!g) return;
  const float2* q = qsum + blockIdx.x * NN;
  float2* o = g + blockIdx.x * NN;
  if (!FAR) {
    for (size_t i = threadIdx.x; i < NN; i += NT) o[i] = cadd(o[i], q[i]);
    return;
  }
  F::fill_twiddles(tw, twg);
  __syncthreads();
  const float invNN = 1.0f / (float)NN;
  using V1 = float2[N1];
  using V2 = float2[N2];
  pass_r23<N, 0, +1>(A, tw, [&](V2& v, int ky, int t) {
#pragma unroll
    for (int i = 0; i < N2; ++i) v[i] = cscale(q[ky * N + t + N1 * i], invNN);
  });
  __syncthreads();
  pass_r14<N, false, +1>(A, tw);
  __syncthreads();
  pass_c23<N, true, +1>(A, tw);
  __syncthreads();
  pass_c14<N, +1, 0, true, false>(A, tw, NoPre(), [&](V1& v, V1&, V1&, int x, int t) {
#pragma unroll
    for (int k = 0; k < N1; ++k) {
      const int p = (N2 * k + t) * N + x;
      o[p] = cadd(o[p], v[k]);
    }
  });
}

// ---------------------------------------------------------------------------- launchers
int path_smem_bytes(int N) {
  switch (N) {
    case 8: return path_smem_bytes_t<8>();
    case 16: return path_smem_bytes_t<16>();
    case 32: return path_smem_bytes_t<32>();
    case 64: return path_smem_bytes_t<64>();
    case 128: return path_smem_bytes_t<128>();
    default: return 0;
  }
}

cudaError_t launch_path(const PathArgs& a, int farfield, cudaStream_t s) {
  if (a.hyj) return launch_path_gaps(a, farfield, s);   // variable slice spacing
  if (a.pipe) return launch_path_pipe(a, farfield, s);
  if (a.helpers) return launch_path_help(a, farfield, s);
  switch (a.N) {
#define ADORYM_CASE(n)                                                                      \
  case n:                                                                                   \
    return farfield ? launch_path_t<n, 1, false>(a, s) : launch_path_t<n, 0, false>(a, s);
    ADORYM_CASE(8)
    ADORYM_CASE(16)
    ADORYM_CASE(32)
    ADORYM_CASE(64)
    ADORYM_CASE(128)
#undef ADORYM_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <int N>
static cudaError_t launch_probe_hat_t(int M, const float2* probe, float2* phat, const float2* tw, cudaStream_t s) {
  const int smem = (N * (N + 1) + Field<N>::TW_ENTRIES) * (int)sizeof(float2);
  (k_probe_hat<N><<<M, Geo<N>::NT, smem, s>>>(probe, phat, tw), note_launch());
  return cudaGetLastError();
}

cudaError_t launch_probe_hat(int N, int M, const float2* probe, float2* phat, const float2* tw, cudaStream_t s) {
  switch (N) {
    case 8: return launch_probe_hat_t<8>(M, probe, phat, tw, s);
    case 16: return launch_probe_hat_t<16>(M, probe, phat, tw, s);
    case 32: return launch_probe_hat_t<32>(M, probe, phat, tw, s);
    case 64: return launch_probe_hat_t<64>(M, probe, phat, tw, s);
    case 128: return launch_probe_hat_t<128>(M, probe, phat, tw, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int N, int FAR>
static cudaError_t launch_probe_grad_t(int M, int B, const float2* qacc, float2* qsum, float2* g, const float2* tw,
                                       const double* lossp, double inv_npix, double* loss_out, cudaStream_t s) {
  const size_t MNN = (size_t)M * N * N;
  if (g) {
    (k_qsum<<<(unsigned)((MNN + 31) / 32), 256, 0, s>>>(qacc, qsum, B, MNN), note_launch());
  }
  const int smem = (N * (N + 1) + Field<N>::TW_ENTRIES) * (int)sizeof(float2);
  (k_probe_grad<N, FAR><<<M, Geo<N>::NT, smem, s>>>(qsum, g, tw, lossp, B, inv_npix, loss_out), note_launch());
  return cudaGetLastError();
}

cudaError_t launch_probe_grad(int N, int M, int B, int farfield, const float2* qacc, float2* qsum, float2* g_probe,
                              const float2* tw, const double* lossp, double inv_npix, double* loss_out,
                              cudaStream_t s) {
  switch (N) {
#define ADORYM_CASE(n)                                                                                     \
  case n:                                                                                                  \
    return farfield ? launch_probe_grad_t<n, 1>(M, B, qacc, qsum, g_probe, tw, lossp, inv_npix, loss_out, s) \
                    : launch_probe_grad_t<n, 0>(M, B, qacc, qsum, g_probe, tw, lossp, inv_npix, loss_out, s);
    ADORYM_CASE(8)
    ADORYM_CASE(16)
    ADORYM_CASE(32)
    ADORYM_CASE(64)
    ADORYM_CASE(128)
#undef ADORYM_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <int N, int FAR>
static cudaError_t prepare_t() {
  cudaError_t e = prepare_path_t<N, FAR, false>();
  if (e == cudaSuccess) e = prepare_path_gaps(N, FAR);
  if (e == cudaSuccess) e = prepare_path_pipe(N, FAR);
  if (e == cudaSuccess) e = prepare_path_help(N, FAR);
  const int small = (N * (N + 1) + Field<N>::TW_ENTRIES) * (int)sizeof(float2);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_probe_hat<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, small);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_probe_grad<N, FAR>, cudaFuncAttributeMaxDynamicSharedMemorySize, small);
  return e;
}

cudaError_t prepare_path(int N, int farfield) {
  // idempotent; called by every entry point before it enqueues (never inside a stream capture)
  static std::atomic<bool> done[kMaxDevices][11][2] = {};
  const int dev = current_device();
  int l = 0;
  while ((1 << l) < N) ++l;
  if (dev >= 0 && l < 11 && done[dev][l][farfield ? 1 : 0].load(std::memory_order_acquire)) return cudaSuccess;
  cudaError_t e = cudaErrorInvalidValue;
  switch (N) {
#define ADORYM_CASE(n) \
  case n:              \
    e = farfield ? prepare_t<n, 1>() : prepare_t<n, 0>(); \
    break;
    ADORYM_CASE(8)
    ADORYM_CASE(16)
    ADORYM_CASE(32)
    ADORYM_CASE(64)
    ADORYM_CASE(128)
#undef ADORYM_CASE
    default:
      return cudaErrorInvalidValue;
  }
  if (e == cudaSuccess && dev >= 0 && l < 11) done[dev][l][farfield ? 1 : 0].store(true, std::memory_order_release);
  return e;
}

}  // namespace adorym
