// Fused multislice forward + loss + adjoint, one CTA per position (far field) or per problem
// (near field), wavefield resident in shared memory (N <= 128).
//
// Forward (Algorithm 1, per probe mode):
//   psi_0   = IDFT_-{ DFT_-[P] exp(-2 pi i dr.nu) }                 Eq. fourier_shift
//   phi_j   = psi_j exp(-k dz beta_j) exp(i k dz delta_j)           Eq. ri_modulation
//   psi_j+1 = IDFT_-{ DFT_-[phi_j] H },  H = exp(i pi lambda dz |nu|^2)   Eqs. fresnel_prop, paraxial_kernel
//   far:  Psi = (1/N) DFT_+[phi_L-1]                                 Eq. fraunhofer (negative phase convention)
//   near: Psi_d = IDFT_-{ DFT_-[phi_L-1] H_d exp(-2 pi i s_d.nu) }   Eq. fresnel_prop to the detector
//   I = sum_modes |Psi|^2                                            Eq. multimode
// Loss: mean over the batch's detector pixels of Eq. lsq_loss (amplitudes, I + eps) or
// Eq. poisson_loss (log(I + eps)), summed Kahan-compensated per thread and in FP64 across threads.
// Adjoint (chain rule; the paper obtains it by reverse-mode AD, Sec. 2.3.1):
//   Psibar = 2 dL/dI Psi;  phibar_L-1 = (1/N) DFT_-[Psibar] (far) or IDFT_-{sum_d conj(G_d) DFT_-[Psibar_d]} (near)
//   psibar_j = conj(T_j) phibar_j;  dL/ddelta_j += k dz Im(psibar_j conj psi_j);
//   dL/dbeta_j += -k dz Re(psibar_j conj psi_j);  phibar_j-1 = IDFT_-{ DFT_-[psibar_j] conj H }
//   far: Q = DFT_-[psibar_0];  dL/dP = IDFT_-{ sum_b Q conj(ramp) } (reduced later);
//        dL/ddr_a = Re[(1/N^2) sum_nu conj(Q) (-2 pi i nu_a) P^ ramp]
//   near: dL/dP = sum_b psibar_0;  dL/ds_d,a = Re[(1/N^2) sum_nu conj(Q_d) (-2 pi i nu_a) Phi G_d]
// The psi_j needed by the adjoint are not kept: psi is checkpointed every cp slices
// (cp = ceil(sqrt(L)) by default) and each segment is recomputed from its checkpoint
// before it is reversed (the recompute-vs-store trade-off discussed in Sec. 4).
//
// Pipelined variant (PIPE, batches of at most half the SM count): each position gets a cluster of
// two CTAs.  Rank 0 runs the forward, the loss and the adjoint sweep; rank 1 recomputes segment
// s-1 from its checkpoint while rank 0 reverses segment s, into the other half of a
// double-buffered segment store, so the recompute leaves the critical path.  The two meet at one
// hardware cluster barrier per segment (no spin-waits).
//
// Recompute helpers (one CTA per position, batch below the SM count): the SMs the batch leaves
// idle run helper CTAs that recompute segments 0, 1, ... of every position (in that order: the
// adjoint sweep needs them last, and their checkpoints are written first) into a separate store.
// A position takes each segment with an atomic compare-and-swap when its sweep reaches it: a
// segment no helper has started is recomputed by the position itself, a finished one is read from
// the store, and only a segment a helper is working on is waited for.  A helper waits for a
// checkpoint only before claiming its segment.  Both waits are bounded (a helper skips the
// segment, a position recomputes it itself), so no CTA depends on another being resident.
#pragma once
#include "numerics.cuh"
#include "fft_block.cuh"
#include "fft_block4.cuh"
#include "kernels.cuh"

namespace adorym {

template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < NT / 32; ++i) s += red[i];   // fixed order: deterministic
  }
  __syncthreads();
  return s;   // valid on thread 0
}

// frequency f_k of bin k in cycles per pixel (Nyquist bin negative), exact in FP32 (N a power of two)
__device__ __forceinline__ float freqf1(int k, int N) { return (float)(k <= (N - 1) / 2 ? k : k - N) * (1.0f / (float)N); }

// exp(-2 pi i d f_k) for k < N into out (d exact in FP32: a float shift, or a float position
// minus its integer corner)
__device__ __forceinline__ void ramp_table(float2* out, float d, int N, int NT) {
  for (int k = threadIdx.x; k < N; k += NT) out[k] = shift_ramp(d, k, N);
}

// both CTAs of a cluster arrive, then wait: global and shared writes made before the barrier by
// either CTA are visible to both after it
__device__ __forceinline__ void cluster_barrier() {
  __threadfence();
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// gpu-scope acquire load / release store of a flag word (helper protocol)
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// thread 0 of a position's CTA at segment s: take the segment (0 -> 3) or find it recomputed by a
// helper.  Waits, bounded by `limit` cycles (about 2^28 by default), only while a helper holds it
// (1).  True: the helper's slices are complete and visible; false: the position recomputes the
// segment itself.
__device__ __forceinline__ bool take_segment(int* flag, long long limit) {
  int st = atomicCAS(flag, 0, 3);
  if (st == 1) {
    const long long t0 = clock64();
    do {
      __nanosleep(256);
      st = ld_acquire_gpu(flag);
    } while (st == 1 && clock64() - t0 < limit);
  }
  __threadfence();
  return st == 2;
}

// thread 0 of a helper: wait until the position's forward has written `need` checkpoints (1);
// 0 when the position took the segment meanwhile; -1 after `limit` cycles (about 2^24 by default:
// the position is not progressing, e.g. not resident, and the helper stops so that it does not
// hold the SM)
__device__ __forceinline__ int wait_checkpoints(const int* prog, int need, const int* flag, long long limit) {
  const long long t0 = clock64();
  for (;;) {
    if (ld_acquire_gpu(prog) >= need) return 1;
    if (*reinterpret_cast<const volatile int*>(flag) != 0) return 0;
    if (clock64() - t0 > limit) return -1;
    __nanosleep(512);
  }
}

// GAP: per-gap propagators (variable slice spacing) and the slice-gap gradient; the uniform-spacing
// instantiation carries none of that code.  PIPE: the two-CTA cluster form described above.
// HELP: the position side of the recompute-helper protocol (a separate instantiation, so that
// calls without helpers run code with the register allocation of the plain form).
template <int N, int FAR, bool GAP, bool PIPE, bool HELP = false>
__device__ __forceinline__ void path_body(const PathArgs& a) {
  static_assert(!(HELP && (GAP || PIPE)), "recompute helpers serve the plain one-CTA form only");
  using F = Field<N>;
  using X = PathFFT<N>;
  constexpr int CY = X::CY, YS = X::YS, RX = X::RX, KXS = X::KXS, LD = F::LD, NT = F::NT;
  constexpr size_t NN = (size_t)N * N;
  using V1 = float2[CY];
  using V2 = float2[RX];
  extern __shared__ float2 sm[];
  float2* A = sm;
  float2* tw = A + N * LD;             // F::TW_ENTRIES twiddles (tw, then the per-stage tables)
  float2* hy = tw + F::TW_ENTRIES;
  float2* hx = hy + N;
  float2* ry = hx + N;
  float2* rx = ry + N;
  double* red = reinterpret_cast<double*>(rx + N);

  static_assert(!(GAP && PIPE), "the pipelined form has no slice-gap gradient");
  const int b = PIPE ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int rank = PIPE ? (int)(blockIdx.x & 1) : 0;   // cluster of two CTAs along x
  const int M = a.M, L = a.L, cp = a.cp, ncp = a.ncp;
  F::fill_twiddles(tw, a.tw);
  for (int i = threadIdx.x; i < N; i += NT) {
    hy[i] = a.hy[i];
    hx[i] = a.hx[i];
  }
  int p0y = 0, p0x = 0;
  if (FAR) {
    // S1: integer corner p0 = floor(pos + 1/2), residual dr = pos - p0 (FP64, exact for float input)
    const double py = a.pos[2 * b], px = a.pos[2 * b + 1];
    const double fy = floor(py + 0.5), fx = floor(px + 0.5);
    p0y = patch_corner(a.pos[2 * b]);
    p0x = patch_corner(a.pos[2 * b + 1]);
    ramp_table(ry, (float)(py - fy), N, NT);
    ramp_table(rx, (float)(px - fx), N, NT);
  }
  __syncthreads();

  const int Ly = a.Ly, Lx = a.Lx;
  const float kdz = a.kdz;
  int cur_mode = 0;   // probe mode being processed (partials of mode 0 overwrite, later modes add)
  // transmission T_j at patch pixel (y, x); voxels outside the volume are vacuum (T = 1).  A patch
  // that lies inside the volume (the usual case; CTA-uniform) skips the per-pixel bounds tests.
  const bool interior = p0y >= 0 && p0x >= 0 && p0y <= Ly - N && p0x <= Lx - N;
  const size_t slab = (size_t)Ly * Lx;
  auto tload = [&](int j, int y, int x) -> float2 {
    const int gy = p0y + y, gx = p0x + x, gz = FAR ? j : b * L + j;
    if (gy >= 0 && gy < Ly && gx >= 0 && gx < Lx) return __ldg(a.T + ((size_t)gz * Ly + gy) * Lx + gx);
    return make_float2(1.f, 0.f);
  };
  // offset of patch pixel (t, x) of slice j in the volume (interior patches)
  auto voff = [&](int j, int t, int x) -> size_t {
    return (size_t)(FAR ? j : b * L + j) * slab + (size_t)(p0y + t) * Lx + (p0x + x);
  };
  auto tloads = [&](V1& pa, int j, int x, int t) {
    if (interior) {
      const float2* p = a.T + voff(j, t, x);
#pragma unroll
      for (int k = 0; k < CY; ++k) pa[k] = __ldg(p + (size_t)(YS * k) * Lx);
    } else {
#pragma unroll
      for (int k = 0; k < CY; ++k) pa[k] = tload(j, YS * k + t, x);
    }
  };
  auto pre_T = [&](int j) {
    return [&, j](V1& pa, V1&, int x, int t) { tloads(pa, j, x, t); };
  };
  // the rest of a propagation step after C14: C2, R1, R23(H_gap or conj H_gap), R4, C3.  With
  // variable spacing (GAP) the propagator factors of gap `gapj` come from the per-gap tables;
  // spec_out keeps F[psi_{gapj+1}] / N^2 for the slice-gap gradient, spec_in (adjoint)
  // accumulates dL/dc_gap = -pi sum |f|^2 Im(conj(F[psibar]) F[psi]) into gapp
  auto propagate_tail = [&](bool adjoint, int gapj, float2* spec_out, const float2* spec_in) {
    X::template fwd_pair<-1>(A, tw);
    __syncthreads();
    float gs = 0.f;
    if constexpr (GAP) {
      const float2* hyp = a.hyj + (size_t)gapj * N;
      const float2* hxp = a.hxj + (size_t)gapj * N;
      X::template r23<-1, +1>(A, tw, [&](V2& v, int ky, int t) {
        const float2 h = hyp[ky];
        const float fy = freqf1(ky, N);
#pragma unroll
        for (int i = 0; i < RX; ++i) {
          const int kx = t + KXS * i;
          const float2 H = cmul(h, hxp[kx]);
          if (!adjoint) {
            v[i] = cmul(v[i], H);
            if (spec_out) spec_out[ky * N + kx] = v[i];
          } else {
            if (spec_in) {
              const float fx = freqf1(kx, N);
              gs += (fy * fy + fx * fx) * cmulc(spec_in[ky * N + kx], v[i]).y;
            }
            v[i] = cmulc(v[i], H);
          }
        }
      });
    } else if (adjoint) {
      X::template r23<-1, +1>(A, tw, [&](V2& v, int ky, int t) {
        const float2 h = hy[ky];
#pragma unroll
        for (int i = 0; i < RX; ++i) v[i] = cmulc(cmulc(v[i], h), hx[t + KXS * i]);
      });
    } else {
      X::template r23<-1, +1>(A, tw, [&](V2& v, int ky, int t) {
        const float2 h = hy[ky];
#pragma unroll
        for (int i = 0; i < RX; ++i) v[i] = cmul(cmul(v[i], h), hx[t + KXS * i]);
      });
    }
    __syncthreads();
    X::template inv_pair<+1>(A, tw);
    __syncthreads();
    if constexpr (GAP) {
      if (adjoint && spec_in) {
        const double g = block_sum<NT>(f32_to_f64(gs), red);
        if (threadIdx.x == 0) {
          double* gp = a.gapp + (size_t)blockIdx.x * (a.L - 1) + gapj;
          const double val = -3.14159265358979323846 * g;
          *gp = (cur_mode == 0) ? val : *gp + val;
        }
      }
    }
  };

  const bool adj = a.adj != 0;
  const int nd = FAR ? 1 : a.n_dist;
  const int j0_last = (ncp - 1) * cp;
  const float invN = 1.0f / (float)N, invNN = 1.0f / (float)NN;
  float2* ck_b = a.ckpt + (size_t)b * M * ncp * NN;
  // segment store: one set of cp slices per (b, m), two in the pipelined form (slot = s % 2)
  constexpr int NSLOT = PIPE ? 2 : 1;
  float2* seg_b = a.seg + (size_t)b * M * NSLOT * cp * NN;
  auto seg_slot = [&](int m, int s) -> float2* {
    return seg_b + ((size_t)m * NSLOT + (PIPE ? (s & 1) : 0)) * cp * NN;
  };
  float* gI_b = a.gI + (size_t)b * nd * NN;

  const bool want_gap = GAP && adj && a.gapp != nullptr;
  float2* spck_b = want_gap ? a.spck + (size_t)b * M * ncp * NN : nullptr;
  float2* spsg_b = want_gap ? a.spseg + (size_t)b * M * cp * NN : nullptr;
  if (rank == 0) {
  // ------------------------------------------------------------------ forward
  for (int m = 0; m < M; ++m) {
    cur_mode = m;
    float2* ck = ck_b + (size_t)m * ncp * NN;
    float2* sg = seg_slot(m, ncp - 1);   // the last segment is kept by the forward pass
    float2* spck = want_gap ? spck_b + (size_t)m * ncp * NN : nullptr;
    float2* spsg = want_gap ? spsg_b + (size_t)m * cp * NN : nullptr;
    // spectrum slot of slice jn (propagated into by gap jn - 1): checkpoint or last segment
    auto spec_slot_fwd = [&](int jn) -> float2* {
      if (!want_gap) return nullptr;
      if (jn % cp == 0) return spck + (size_t)(jn / cp) * NN;
      if (jn > j0_last) return spsg + (size_t)(jn - j0_last) * NN;
      return nullptr;
    };
    // spatial op of slice j: store psi_j where the adjoint needs it, then modulate.  The slot
    // (checkpoint j / cp, the last segment, or none) is chosen once per slice: decided per pixel,
    // the runtime division by cp made a 128 x 128 forward step 13.8 instead of 10.9 us.
    auto fwd_op = [&](int j, bool from_pb) {
      float2* keep = !adj ? nullptr
                     : (j % cp == 0) ? ck + (size_t)(j / cp) * NN
                     : (j > j0_last) ? sg + (size_t)(j - j0_last) * NN
                                     : nullptr;
      return [&, keep, from_pb](V1& v, V1& pa, V1& pb, int x, int t) {
#pragma unroll
        for (int k = 0; k < CY; ++k) {
          const int y = YS * k + t;
          if (from_pb) v[k] = pb[k];
          if (keep) keep[y * N + x] = v[k];
          v[k] = cmul(v[k], pa[k]);
        }
      };
    };
    if (FAR) {
      // psi_0 = IDFT_-(P^ ramp), built in Fourier space at the R23 layout
      const float2* ph = a.phat + (size_t)m * NN;
      X::template r23<0, +1>(A, tw, [&](V2& v, int ky, int t) {
        const float2 r = cscale(ry[ky], invNN);
#pragma unroll
        for (int i = 0; i < RX; ++i) {
          const int kx = t + KXS * i;
          v[i] = cmul(cmul(__ldg(&ph[ky * N + kx]), r), rx[kx]);
        }
      });
      __syncthreads();
      X::template inv_pair<+1>(A, tw);
      __syncthreads();
    }
    for (int j = 0; j < L; ++j) {
      const bool last = (j == L - 1);
      if (!FAR && j == 0) {
        // the illumination enters through pb; near field always starts its last transform with DFT_-
        const float2* pr = a.probe + (size_t)m * NN;
        auto T0 = pre_T(0);
        X::template c14<0, -1, false, true>(A, tw, [&](V1& pa, V1& pb, int x, int t) {
          T0(pa, pb, x, t);
#pragma unroll
          for (int k = 0; k < CY; ++k) pb[k] = __ldg(&pr[(YS * k + t) * N + x]);
        }, fwd_op(0, true));
      } else if (FAR && last) {
        X::template c14<+1, +1, true, true>(A, tw, pre_T(j), fwd_op(j, false));
      } else {
        X::template c14<+1, -1, true, true>(A, tw, pre_T(j), fwd_op(j, false));
      }
      __syncthreads();
      if constexpr (HELP) {
        // checkpoint j / cp is written: helpers may recompute segment j / cp from now on
        if (a.helpers && adj && j % cp == 0 && threadIdx.x == 0) {
          __threadfence();
          st_release_gpu(a.hprog + (size_t)b * M + m, j / cp + 1);
        }
      }
      if (!last) {
        propagate_tail(false, j, spec_slot_fwd(j + 1), nullptr);
        continue;
      }
      if (FAR) {
        // Psi = (1/N) DFT_+[phi]; keep Psi, accumulate I over modes
        X::template fwd_pair<+1>(A, tw);
        __syncthreads();
        float2* fm = a.far + ((size_t)b * M + m) * NN;
        X::template r23<+1, 0>(A, tw, [&](V2& v, int ky, int t) {
#pragma unroll
          for (int i = 0; i < RX; ++i) {
            const int p = ky * N + t + KXS * i;
            const float2 P = cscale(v[i], invN);
            fm[p] = P;
            const float I = fmaf(P.x, P.x, P.y * P.y);
            gI_b[p] = (m == 0) ? I : gI_b[p] + I;
          }
        });
        __syncthreads();
      } else {
        // Phi = DFT_-[phi] kept at slot n_dist; then Psi_d = IDFT_-{Phi G_d} per distance
        X::template fwd_pair<-1>(A, tw);
        __syncthreads();
        float2* Phi = a.far + (((size_t)b * (nd + 1) + nd) * M + m) * NN;
        X::template r23<-1, 0>(A, tw, [&](V2& v, int ky, int t) {
#pragma unroll
          for (int i = 0; i < RX; ++i) Phi[ky * N + t + KXS * i] = v[i];
        });
        __syncthreads();
        for (int d = 0; d < nd; ++d) {
          const float* sd = a.pos + ((size_t)b * nd + d) * 2;
          ramp_table(ry, sd[0], N, NT);
          ramp_table(rx, sd[1], N, NT);
          __syncthreads();
          const float2* hd = a.hd + (size_t)d * N;
          X::template r23<0, +1>(A, tw, [&](V2& v, int ky, int t) {
            const float2 gy = cscale(cmul(__ldg(&hd[ky]), ry[ky]), invNN);
#pragma unroll
            for (int i = 0; i < RX; ++i) {
              const int kx = t + KXS * i;
              v[i] = cmul(cmul(Phi[ky * N + kx], gy), cmul(__ldg(&hd[kx]), rx[kx]));
            }
          });
          __syncthreads();
          X::template inv_pair<+1>(A, tw);
          __syncthreads();
          float2* fd = a.far + (((size_t)b * (nd + 1) + d) * M + m) * NN;
          float* gId = gI_b + (size_t)d * NN;
          X::template c14<+1, 0, true, false>(A, tw, NoPre(), [&](V1& v, V1&, V1&, int x, int t) {
#pragma unroll
            for (int k = 0; k < CY; ++k) {
              const int p = (YS * k + t) * N + x;
              fd[p] = v[k];
              const float I = fmaf(v[k].x, v[k].x, v[k].y * v[k].y);
              gId[p] = (m == 0) ? I : gId[p] + I;
            }
          });
          __syncthreads();
        }
      }
    }
  }

  // ------------------------------------------------------------------ loss, dL/dI
  {
    const size_t npx = (size_t)nd * NN;
    const float* Im = a.I_meas ? a.I_meas + (size_t)b * npx : nullptr;
    float* Io = a.I_out ? a.I_out + (size_t)b * npx : nullptr;
    const float eps = a.eps, sc = (float)a.inv_npix;
    Kahan acc;
    constexpr int U = 4;   // pixels per thread whose loads are issued ahead of their stores
    for (size_t p0 = threadIdx.x; p0 < npx; p0 += (size_t)U * NT) {
      float Iv[U], mv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const size_t p = p0 + (size_t)u * NT;
        Iv[u] = p < npx ? gI_b[p] : 0.f;
        mv[u] = (Im && p < npx) ? __ldg(Im + p) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
      const size_t p = p0 + (size_t)u * NT;
      if (p >= npx) break;
      const float I = Iv[u];
      if (Io) Io[p] = I;
      if (!Im) continue;
      const float im = mv[u];
      float term, dI;
      if (a.loss == 0) {
        const float sI = sqrtf(I + eps), sM = sqrtf(im + eps);
        const float df = sI - sM;
        term = df * df;
        dI = df / sI;
      } else {
        term = I - im * logf(I + eps);
        dI = 1.0f - im / (I + eps);
      }
      acc.add(term);
      gI_b[p] = dI * sc;
      }
    }
    const double s = block_sum<NT>(acc.value(), red);
    if (threadIdx.x == 0 && a.lossp) a.lossp[b] = s;
  }
  }   // rank 0: forward and loss
  if (!adj) return;   // (the pipelined form always runs the adjoint)
  __syncthreads();

  // ------------------------------------------------------------------ adjoint
  double gacc[3 * 4] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};   // per distance: shift y, x; N_F
  const bool want_obj = a.gd != nullptr;   // FP64 accumulators (else a.gdf or nothing)
  for (int m = 0; m < M; ++m) {
    cur_mode = m;
    float2* ck = ck_b + (size_t)m * ncp * NN;
    float2* spck = want_gap ? spck_b + (size_t)m * ncp * NN : nullptr;
    float2* spsg = want_gap ? spsg_b + (size_t)m * cp * NN : nullptr;
    // recompute psi_{j0+1..j1} of segment s from its checkpoint psi_{j0} into segment slot `sg`
    // (the field in shared memory is overwritten)
    auto recompute = [&](int s, float2* sg) {
      const int j0 = s * cp, j1 = min(j0 + cp, L) - 1;
      for (int j = j0; j < j1; ++j) {
        if (j == j0) {
          auto T0 = pre_T(j);
          X::template c14<0, -1, false, true>(A, tw, [&](V1& pa, V1& pb, int x, int t) {
            T0(pa, pb, x, t);
#pragma unroll
            for (int k = 0; k < CY; ++k) pb[k] = __ldcg(ck + (size_t)s * NN + (YS * k + t) * N + x);
          }, [&](V1& v, V1& pa, V1& pb, int, int) {
#pragma unroll
            for (int k = 0; k < CY; ++k) v[k] = cmul(pb[k], pa[k]);
          });
        } else {
          X::template c14<+1, -1, true, true>(A, tw, pre_T(j), [&, j](V1& v, V1& pa, V1&, int x, int t) {
#pragma unroll
            for (int k = 0; k < CY; ++k) {
              sg[(size_t)(j - j0) * NN + (YS * k + t) * N + x] = v[k];
              v[k] = cmul(v[k], pa[k]);
            }
          });
        }
        __syncthreads();
        propagate_tail(false, j, want_gap ? spsg + (size_t)(j + 1 - j0) * NN : nullptr, nullptr);
      }
      X::template c14<+1, 0, true, false>(A, tw, NoPre(), [&](V1& v, V1&, V1&, int x, int t) {
#pragma unroll
        for (int k = 0; k < CY; ++k) sg[(size_t)(j1 - j0) * NN + (YS * k + t) * N + x] = v[k];
      });
      __syncthreads();
    };
    if (PIPE) {
      // checkpoints (and, for m > 0, the previous mode's sweep) are complete
      cluster_barrier();
      if (rank == 1) {
        // recompute segment s - 1 while rank 0 reverses segment s; one barrier per segment
        for (int s = ncp - 1; s >= 0; --s) {
          if (s >= 1 && min((s - 1) * cp + cp, L) - 1 > (s - 1) * cp) recompute(s - 1, seg_slot(m, s - 1));
          cluster_barrier();
        }
        continue;
      }
    }
    if (FAR) {
      // phibar_{L-1} = (1/N) DFT_-[2 gI Psi]
      const float2* fm = a.far + ((size_t)b * M + m) * NN;
      const float sc = 2.0f * invN;
      X::template r23<0, -1>(A, tw, [&](V2& v, int ky, int t) {
#pragma unroll
        for (int i = 0; i < RX; ++i) {
          const int p = ky * N + t + KXS * i;
          v[i] = cscale(fm[p], sc * gI_b[p]);
        }
      });
      __syncthreads();
      X::template inv_pair<-1>(A, tw);
      __syncthreads();
    } else {
      const float2* Phi = a.far + (((size_t)b * (nd + 1) + nd) * M + m) * NN;
      float2* fb = a.fbar + (size_t)b * NN;
      for (int d = 0; d < nd; ++d) {
        const float* sd = a.pos + ((size_t)b * nd + d) * 2;
        ramp_table(ry, sd[0], N, NT);
        ramp_table(rx, sd[1], N, NT);
        const float2* fd = a.far + (((size_t)b * (nd + 1) + d) * M + m) * NN;
        const float* gId = gI_b + (size_t)d * NN;
        __syncthreads();
        // Q_d = DFT_-[2 gI_d Psi_d]
        X::template c14<0, -1, false, true>(A, tw, [&](V1& pa, V1& pb, int x, int t) {
#pragma unroll
          for (int k = 0; k < CY; ++k) {
            const int p = (YS * k + t) * N + x;
            pa[k] = fd[p];
            pb[k].x = gId[p];
          }
        }, [&](V1& v, V1& pa, V1& pb, int, int) {
#pragma unroll
          for (int k = 0; k < CY; ++k) v[k] = cscale(pa[k], 2.0f * pb[k].x);
        });
        __syncthreads();
        X::template fwd_pair<-1>(A, tw);
        __syncthreads();
        const float2* hd = a.hd + (size_t)d * N;
        X::template r23<-1, 0>(A, tw, [&](V2& v, int ky, int t) {
          const float2 gy = cmul(__ldg(&hd[ky]), ry[ky]);
          const float fyk = freqf1(ky, N);
          float ay = 0.f, ax = 0.f, an = 0.f;
#pragma unroll
          for (int i = 0; i < RX; ++i) {
            const int kx = t + KXS * i, p = ky * N + kx;
            const float2 G = cmul(gy, cmul(__ldg(&hd[kx]), rx[kx]));
            const float2 base = cmul(cconj(v[i]), cmul(Phi[p], G));
            const float fxk = freqf1(kx, N);
            ay += fyk * base.y;
            ax += fxk * base.y;
            an += (fyk * fyk + fxk * fxk) * base.y;
            const float2 c = cmulc(v[i], G);   // conj(G) Q
            fb[p] = (d == 0) ? c : cadd(fb[p], c);
          }
          gacc[3 * d] += ay;
          gacc[3 * d + 1] += ax;
          gacc[3 * d + 2] += an;
        });
        __syncthreads();
      }
      // phibar_{L-1} = IDFT_-{sum_d conj(G_d) Q_d}
      X::template r23<0, +1>(A, tw, [&](V2& v, int ky, int t) {
#pragma unroll
        for (int i = 0; i < RX; ++i) v[i] = cscale(fb[ky * N + t + KXS * i], invNN);
      });
      __syncthreads();
      X::template inv_pair<+1>(A, tw);
      __syncthreads();
    }

    for (int s = ncp - 1; s >= 0; --s) {
      const int j0 = s * cp, j1 = min(j0 + cp, L) - 1;
      float2* sg = seg_slot(m, s);
      bool from_helper = false;   // psi_{j0+1..j1} in a helper's store instead of the own slot
      if (!PIPE && s != ncp - 1 && j1 > j0) {
        bool own = true;
        if constexpr (HELP) {
          if (a.helpers) {
            bool done = false;
            if (threadIdx.x == 0) done = take_segment(a.hflag + ((size_t)b * M + m) * ncp + s, a.wait_seg);
            // the vote is CTA-uniform; the lane-0 broadcast lets the compiler treat the branch
            // below as warp-uniform (a plain vote result cost ~6 % through extra spills)
            from_helper = __shfl_sync(0xffffffffu, __syncthreads_or(done), 0) != 0;
            own = !from_helper;
          }
        }
        if (own) {
          // park the adjoint field, recompute the segment in shared memory, restore
          float2* pk = a.park + (size_t)b * N * LD;
          for (int i = threadIdx.x; i < N * LD; i += NT) pk[i] = A[i];
          __syncthreads();
          recompute(s, sg);
          for (int i = threadIdx.x; i < N * LD; i += NT) A[i] = pk[i];
          __syncthreads();
        }
      }
      for (int j = j1; j >= j0; --j) {
        const bool first = (j == 0);
        // prefetch T_j and psi_j (checkpoint or recomputed segment)
        auto pre = [&, j](V1& pa, V1& pb, int x, int t) {
          const float2* seg_j = from_helper ? a.hseg + (((size_t)b * M + m) * (ncp - 1) + s) * cp * NN : sg;
          const float2* src = (j == j0) ? ck + (size_t)s * NN : seg_j + (size_t)(j - j0) * NN;
          tloads(pa, j, x, t);
#pragma unroll
          for (int k = 0; k < CY; ++k) pb[k] = __ldcg(src + (YS * k + t) * N + x);   // L2: written by the partner CTA
        };
        float2* q0 = (!FAR && first && a.qacc) ? a.qacc + ((size_t)b * M + m) * NN : nullptr;
        auto op = [&, j, q0](V1& v, V1& pa, V1& pb, int x, int t) {
          const size_t o0 = interior ? voff(j, t, x) : 0;
#pragma unroll
          for (int k = 0; k < CY; ++k) {
            const int y = YS * k + t;
            const float2 pbar = cmulc(v[k], pa[k]);     // psibar_j = conj(T_j) phibar_j
            if (!FAR && a.gdf) {
              // near field, one mode: this thread owns voxel (b L + j, y, x) for the whole call
              const float2 z = cmulc(pbar, pb[k]);
              const size_t o = voff(j, t, x) + (size_t)(YS * k) * Lx;
              a.gdf[o] += kdz * z.y;
              a.gbf[o] -= kdz * z.x;
            } else if (want_obj) {
              const float2 z = cmulc(pbar, pb[k]);      // psibar conj(psi)
              size_t o = o0 + (size_t)(YS * k) * Lx;
              bool in = interior;
              if (!interior) {
                const int gy = p0y + y, gx = p0x + x, gz = FAR ? j : b * L + j;
                in = gy >= 0 && gy < Ly && gx >= 0 && gx < Lx;
                o = ((size_t)gz * Ly + gy) * Lx + gx;
              }
              if (in) {
                atomicAdd(a.gd + o, f32_to_f64(kdz * z.y));
                atomicAdd(a.gb + o, f32_to_f64(-kdz * z.x));
              }
            }
            v[k] = pbar;
            if (q0) q0[y * N + x] = pbar;               // near field: illumination gradient
          }
        };
        if (FAR && j == L - 1) X::template c14<-1, -1, true, true>(A, tw, pre, op);
        else if (!FAR && first) X::template c14<+1, 0, true, false>(A, tw, pre, op);
        else X::template c14<+1, -1, true, true>(A, tw, pre, op);
        __syncthreads();
        if (!first) {
          const float2* sp_in = !want_gap ? nullptr : (j == j0) ? spck + (size_t)s * NN : spsg + (size_t)(j - j0) * NN;
          propagate_tail(true, j - 1, nullptr, sp_in);
          continue;
        }
        if (!FAR) continue;
        // far field, j = 0: Q = DFT_-[psibar_0] -> probe and position gradients
        X::template fwd_pair<-1>(A, tw);
        __syncthreads();
        const float2* ph = a.phat + (size_t)m * NN;
        float2* q = a.qacc ? a.qacc + ((size_t)b * M + m) * NN : nullptr;
        X::template r23<-1, 0>(A, tw, [&](V2& v, int ky, int t) {
          const float2 r_y = ry[ky];
          const float fyk = freqf1(ky, N);
          float ay = 0.f, ax = 0.f;
#pragma unroll
          for (int i = 0; i < RX; ++i) {
            const int kx = t + KXS * i, p = ky * N + kx;
            const float2 r = cmul(r_y, rx[kx]);
            const float2 base = cmul(cconj(v[i]), cmul(__ldg(&ph[p]), r));
            ay += fyk * base.y;
            ax += freqf1(kx, N) * base.y;
            if (q) q[p] = cmulc(v[i], r);
          }
          gacc[0] += ay;
          gacc[1] += ax;
        });
        __syncthreads();
      }
      if (PIPE) cluster_barrier();   // segment s consumed; rank 1 may overwrite its slot
    }
  }
  if (rank == 0 && (a.gpos || a.gposd || a.gnf)) {
    // dL/ds_a = (2 pi / N^2) sum f_a Im(base);  dL/dN_F = (pi / (N_F^2 N^2)) sum |f|^2 Im(base)
    const double pi = 3.14159265358979323846, sc = 2.0 * pi / (double)NN;
    for (int d = 0; d < nd; ++d) {
      const double gy = block_sum<NT>(gacc[3 * d], red);
      const double gx = block_sum<NT>(gacc[3 * d + 1], red);
      const double gn = FAR ? 0.0 : block_sum<NT>(gacc[3 * d + 2], red);
      if (threadIdx.x == 0) {
        if (a.gpos) {
          a.gpos[((size_t)b * nd + d) * 2] = (float)(sc * gy);
          a.gpos[((size_t)b * nd + d) * 2 + 1] = (float)(sc * gx);
        }
        if (FAR && a.gposd) {
          a.gposd[2 * (size_t)b] = sc * gy;
          a.gposd[2 * (size_t)b + 1] = sc * gx;
        }
        if (!FAR && a.gnf) a.gnf[(size_t)b * nd + d] = (float)(pi * gn / (a.nf[d] * a.nf[d] * (double)NN));
      }
    }
  }
}

// A recompute helper (CTA blockIdx.x >= B of k_path_help): claims segments
// 0..ncp-2 of the positions in segment-major order and recomputes psi_{j0+1..j1} of each from its
// checkpoint into the helper store, with the same passes and operation order as a position's own
// recompute (so the result does not depend on which CTA recomputed a segment).  Kept apart from
// path_body so that the position code keeps its register allocation.
template <int N, int FAR>
__device__ __forceinline__ void helper_body(const PathArgs& a) {
  using F = Field<N>;
  using X = PathFFT<N>;
  constexpr int CY = X::CY, YS = X::YS, RX = X::RX, KXS = X::KXS, LD = F::LD, NT = F::NT;
  constexpr size_t NN = (size_t)N * N;
  using V1 = float2[CY];
  using V2 = float2[RX];
  extern __shared__ float2 sm[];
  float2* A = sm;
  float2* tw = A + N * LD;
  float2* hy = tw + F::TW_ENTRIES;
  float2* hx = hy + N;
  __shared__ int h_task;
  F::fill_twiddles(tw, a.tw);
  for (int i = threadIdx.x; i < N; i += NT) {
    hy[i] = a.hy[i];
    hx[i] = a.hx[i];
  }
  const int M = a.M, L = a.L, cp = a.cp, ncp = a.ncp, B = a.B, Ly = a.Ly, Lx = a.Lx;
  const int MB = M * B, ntask = (ncp - 1) * MB;
  for (;;) {
    if (threadIdx.x == 0) {
      int got = -1;
      for (int tk = atomicAdd(a.hnext, 1); tk < ntask; tk = atomicAdd(a.hnext, 1)) {
        const int s = tk / MB, m = (tk - s * MB) / B, bb = tk - s * MB - m * B;
        if (min(s * cp + cp, L) - 1 <= s * cp) continue;   // one-slice segment: nothing to recompute
        int* fl = a.hflag + ((size_t)bb * M + m) * ncp + s;
        const int w = wait_checkpoints(a.hprog + (size_t)bb * M + m, s + 1, fl, a.wait_ckpt);
        if (w < 0) break;
        if (w > 0 && atomicCAS(fl, 0, 1) == 0) {
          got = tk;
          break;
        }
      }
      h_task = got;
    }
    __syncthreads();   // also orders the table fill and the last task's stores
    const int tk = h_task;
    __syncthreads();
    if (tk < 0) return;
    const int s = tk / MB, m = (tk - s * MB) / B, b = tk - s * MB - m * B;
    const int p0y = FAR ? patch_corner(a.pos[2 * b]) : 0, p0x = FAR ? patch_corner(a.pos[2 * b + 1]) : 0;
    const bool interior = p0y >= 0 && p0x >= 0 && p0y <= Ly - N && p0x <= Lx - N;
    auto tloads = [&](V1& pa, int j, int x, int t) {
      const size_t gz = FAR ? j : (size_t)b * L + j;
      if (interior) {
        const float2* p = a.T + (gz * Ly + (p0y + t)) * Lx + (p0x + x);
#pragma unroll
        for (int k = 0; k < CY; ++k) pa[k] = __ldg(p + (size_t)(YS * k) * Lx);
      } else {
#pragma unroll
        for (int k = 0; k < CY; ++k) {
          const int gy = p0y + YS * k + t, gx = p0x + x;
          pa[k] = (gy >= 0 && gy < Ly && gx >= 0 && gx < Lx) ? __ldg(a.T + (gz * Ly + gy) * Lx + gx)
                                                             : make_float2(1.f, 0.f);
        }
      }
    };
    const size_t bm = (size_t)b * M + m;
    const float2* ck = a.ckpt + (bm * ncp + s) * NN;
    float2* sg = a.hseg + (bm * (ncp - 1) + s) * cp * NN;
    const int j0 = s * cp, j1 = min(j0 + cp, L) - 1;
    for (int j = j0; j < j1; ++j) {
      if (j == j0) {
        X::template c14<0, -1, false, true>(A, tw, [&](V1& pa, V1& pb, int x, int t) {
          tloads(pa, j, x, t);
#pragma unroll
          for (int k = 0; k < CY; ++k) pb[k] = __ldcg(ck + (YS * k + t) * N + x);
        }, [&](V1& v, V1& pa, V1& pb, int, int) {
#pragma unroll
          for (int k = 0; k < CY; ++k) v[k] = cmul(pb[k], pa[k]);
        });
      } else {
        X::template c14<+1, -1, true, true>(A, tw, [&](V1& pa, V1&, int x, int t) { tloads(pa, j, x, t); },
                                        [&](V1& v, V1& pa, V1&, int x, int t) {
#pragma unroll
          for (int k = 0; k < CY; ++k) {
            sg[(size_t)(j - j0) * NN + (YS * k + t) * N + x] = v[k];
            v[k] = cmul(v[k], pa[k]);
          }
        });
      }
      __syncthreads();
      // propagation tail: C2, R1, R23 (H), R4, C3
      X::template fwd_pair<-1>(A, tw);
      __syncthreads();
      X::template r23<-1, +1>(A, tw, [&](V2& v, int ky, int t) {
        const float2 h = hy[ky];
#pragma unroll
        for (int i = 0; i < RX; ++i) v[i] = cmul(cmul(v[i], h), hx[t + KXS * i]);
      });
      __syncthreads();
      X::template inv_pair<+1>(A, tw);
      __syncthreads();
    }
    X::template c14<+1, 0, true, false>(A, tw, NoPre(), [&](V1& v, V1&, V1&, int x, int t) {
#pragma unroll
      for (int k = 0; k < CY; ++k) sg[(size_t)(j1 - j0) * NN + (YS * k + t) * N + x] = v[k];
    });
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      st_release_gpu(a.hflag + bm * ncp + s, 2);
    }
  }
}

template <int N, int FAR, bool GAP>
__global__ void __launch_bounds__(Geo<N>::NT, Geo<N>::MINB) k_path(const PathArgs a) {
  path_body<N, FAR, GAP, false>(a);
}

// with recompute helpers: grid B + helpers, CTAs beyond the batch are helpers
template <int N, int FAR>
__global__ void __launch_bounds__(Geo<N>::NT, Geo<N>::MINB) k_path_help(const PathArgs a) {
  if ((int)blockIdx.x >= a.B) {
    helper_body<N, FAR>(a);
    return;
  }
  path_body<N, FAR, false, false, true>(a);
}

// the pipelined form: grid 2 B, clusters of two CTAs (rank 0 adjoint, rank 1 recompute)
template <int N, int FAR>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(Geo<N>::NT, Geo<N>::MINB) k_path_pipe(const PathArgs a) {
  path_body<N, FAR, false, true>(a);
}

// field + twiddle tables (3N) + hy, hx, ry, rx tables + one double per warp for block reductions
template <int N>
constexpr int path_smem_bytes_t() {
  return (N * (N + 1) + Field<N>::TW_ENTRIES + 4 * N) * (int)sizeof(float2) + (Geo<N>::NT / 32) * (int)sizeof(double);
}

template <int N, int FAR, bool GAP>
cudaError_t launch_path_t(const PathArgs& a, cudaStream_t s) {
  (k_path<N, FAR, GAP><<<a.B, Geo<N>::NT, path_smem_bytes_t<N>(), s>>>(a), note_launch());
  return cudaGetLastError();
}

template <int N, int FAR>
cudaError_t launch_path_help_t(const PathArgs& a, cudaStream_t s) {
  // positions, then the recompute helpers
  (k_path_help<N, FAR><<<a.B + a.helpers, Geo<N>::NT, path_smem_bytes_t<N>(), s>>>(a), note_launch());
  return cudaGetLastError();
}

template <int N, int FAR>
cudaError_t launch_path_pipe_t(const PathArgs& a, cudaStream_t s) {
  (k_path_pipe<N, FAR><<<2 * a.B, Geo<N>::NT, path_smem_bytes_t<N>(), s>>>(a), note_launch());
  return cudaGetLastError();
}

template <int N, int FAR, bool GAP>
cudaError_t prepare_path_t() {
  return cudaFuncSetAttribute(k_path<N, FAR, GAP>, cudaFuncAttributeMaxDynamicSharedMemorySize, path_smem_bytes_t<N>());
}

template <int N, int FAR>
cudaError_t prepare_path_help_t() {
  return cudaFuncSetAttribute(k_path_help<N, FAR>, cudaFuncAttributeMaxDynamicSharedMemorySize, path_smem_bytes_t<N>());
}

template <int N, int FAR>
cudaError_t prepare_path_pipe_t() {
  return cudaFuncSetAttribute(k_path_pipe<N, FAR>, cudaFuncAttributeMaxDynamicSharedMemorySize, path_smem_bytes_t<N>());
}

}  // namespace adorym
