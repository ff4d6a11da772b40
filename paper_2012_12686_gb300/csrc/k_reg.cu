// Regularizers of Table regularizers in the refractive-index form, added to the data term as in
// Eq. tikhonov:
//   R = (1/N_o) [ sum a_d W_d |delta| + a_b W_b |beta| + gamma sum_axes (|grad delta| + |grad beta|) ]
// with forward differences (no term past the last index), subgradient 0 at 0, and optional
// reweighting W = max|C| / (|C| + eps) from a snapshot.  Dense volume work, HBM-bound: one pass
// reads delta, beta (and W), each voxel gathers its own TV subgradient from its neighbours (no
// atomics), per-CTA FP64 partial sums are added in a fixed order.
#include <algorithm>
#include <cstdint>

#include "numerics.cuh"
#include "kernels.cuh"

namespace adorym {

__device__ __forceinline__ float sgn(float v) { return (v > 0.f) - (v < 0.f); }

// One CTA per volume row (z, y) at a time (grid-stride over rows), threads along x: coalesced
// loads, row and plane neighbours from L1/L2, and no per-voxel 64-bit index division.
template <bool TV>
__global__ void __launch_bounds__(256) k_regularize(const float* __restrict__ d, const float* __restrict__ b,
                                                    const float* __restrict__ wd, const float* __restrict__ wb,
                                                    int Lz, int Ly, int Lx, float ad, float ab, float gam,
                                                    float invNo, float* __restrict__ gd, float* __restrict__ gb,
                                                    double* __restrict__ part) {
  __shared__ double red[8];
  const size_t sy = Lx, sz = (size_t)Lx * Ly;
  const int rows = Ly * Lz;
  Kahan acc;
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    const int z = r / Ly, y = r - z * Ly;
    const size_t base = (size_t)r * Lx;
    for (int x = threadIdx.x; x < Lx; x += blockDim.x) {
      const size_t i = base + x;
      const float vd = d[i], vb = b[i];
      const float w1 = wd ? wd[i] : 1.f, w2 = wb ? wb[i] : 1.f;
      float term = ad * w1 * fabsf(vd) + ab * w2 * fabsf(vb);
      float g1 = ad * w1 * sgn(vd), g2 = ab * w2 * sgn(vb);
      if (TV) {
        const int pos[3] = {x, y, z}, lim[3] = {Lx, Ly, Lz};
        const size_t st[3] = {1, sy, sz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (pos[a] + 1 < lim[a]) {
            const float fd = d[i + st[a]] - vd, fb = b[i + st[a]] - vb;
            term += gam * (fabsf(fd) + fabsf(fb));
            g1 -= gam * sgn(fd);
            g2 -= gam * sgn(fb);
          }
          if (pos[a] > 0) {
            g1 += gam * sgn(vd - d[i - st[a]]);
            g2 += gam * sgn(vb - b[i - st[a]]);
          }
        }
      }
      acc.add(term);
      if (gd) {
        gd[i] += g1 * invNo;
        gb[i] += g2 * invNo;
      }
    }
  }
  double v = acc.value();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += red[k];
    part[blockIdx.x] = s;
  }
}

// The same value and gradient with four consecutive voxels of a row per thread (Lx % 4 == 0 and
// 16-byte aligned arrays): 128-bit loads of delta, beta, the weights, the neighbour rows and
// planes and the gradients, the x neighbours across the group from two scalar loads.  Same
// per-voxel arithmetic and the same Kahan order within a thread as k_regularize.
template <bool TV>
__global__ void __launch_bounds__(256) k_regularize4(const float* __restrict__ d, const float* __restrict__ b,
                                                     const float* __restrict__ wd, const float* __restrict__ wb,
                                                     int Lz, int Ly, int Lx, float ad, float ab, float gam,
                                                     float invNo, float* __restrict__ gd, float* __restrict__ gb,
                                                     double* __restrict__ part) {
  __shared__ double red[8];
  const int Lx4 = Lx >> 2;
  const size_t sy = Lx, sz = (size_t)Lx * Ly;
  const size_t n4 = (size_t)Ly * Lz * Lx4;
  const float4 one4 = make_float4(1.f, 1.f, 1.f, 1.f);
  Kahan acc;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(q / Lx4), x0 = 4 * (int)(q - (size_t)r * Lx4);
    const int z = r / Ly, y = r - z * Ly;
    const size_t i = (size_t)r * Lx + x0;
    const float4 vd = *reinterpret_cast<const float4*>(d + i), vb = *reinterpret_cast<const float4*>(b + i);
    const float4 w1 = wd ? *reinterpret_cast<const float4*>(wd + i) : one4;
    const float4 w2 = wb ? *reinterpret_cast<const float4*>(wb + i) : one4;
    const float cd[4] = {vd.x, vd.y, vd.z, vd.w}, cb[4] = {vb.x, vb.y, vb.z, vb.w};
    const float cw1[4] = {w1.x, w1.y, w1.z, w1.w}, cw2[4] = {w2.x, w2.y, w2.z, w2.w};
    float term[4], g1[4], g2[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      term[e] = ad * cw1[e] * fabsf(cd[e]) + ab * cw2[e] * fabsf(cb[e]);
      g1[e] = ad * cw1[e] * sgn(cd[e]);
      g2[e] = ab * cw2[e] * sgn(cb[e]);
    }
    if (TV) {
      // x neighbours: within the group, and one scalar on each side
      float nd[6], nb[6];   // nd[e + 1] = delta at x0 + e, e = -1..4
      nd[0] = x0 > 0 ? d[i - 1] : 0.f;
      nb[0] = x0 > 0 ? b[i - 1] : 0.f;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        nd[e + 1] = cd[e];
        nb[e + 1] = cb[e];
      }
      nd[5] = x0 + 4 < Lx ? d[i + 4] : 0.f;
      nb[5] = x0 + 4 < Lx ? b[i + 4] : 0.f;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int x = x0 + e;
        if (x + 1 < Lx) {
          const float fd = nd[e + 2] - cd[e], fb = nb[e + 2] - cb[e];
          term[e] += gam * (fabsf(fd) + fabsf(fb));
          g1[e] -= gam * sgn(fd);
          g2[e] -= gam * sgn(fb);
        }
        if (x > 0) {
          g1[e] += gam * sgn(cd[e] - nd[e]);
          g2[e] += gam * sgn(cb[e] - nb[e]);
        }
      }
      // y and z neighbours: whole groups of the adjacent rows and planes
      const int pos[2] = {y, z}, lim[2] = {Ly, Lz};
      const size_t st[2] = {sy, sz};
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        if (pos[a] + 1 < lim[a]) {
          const float4 ud = *reinterpret_cast<const float4*>(d + i + st[a]);
          const float4 ub = *reinterpret_cast<const float4*>(b + i + st[a]);
          const float qd[4] = {ud.x, ud.y, ud.z, ud.w}, qb[4] = {ub.x, ub.y, ub.z, ub.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float fd = qd[e] - cd[e], fb = qb[e] - cb[e];
            term[e] += gam * (fabsf(fd) + fabsf(fb));
            g1[e] -= gam * sgn(fd);
            g2[e] -= gam * sgn(fb);
          }
        }
        if (pos[a] > 0) {
          const float4 ud = *reinterpret_cast<const float4*>(d + i - st[a]);
          const float4 ub = *reinterpret_cast<const float4*>(b + i - st[a]);
          const float qd[4] = {ud.x, ud.y, ud.z, ud.w}, qb[4] = {ub.x, ub.y, ub.z, ub.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            g1[e] += gam * sgn(cd[e] - qd[e]);
            g2[e] += gam * sgn(cb[e] - qb[e]);
          }
        }
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) acc.add(term[e]);
    if (gd) {
      float4 od = *reinterpret_cast<float4*>(gd + i), ob = *reinterpret_cast<float4*>(gb + i);
      od.x += g1[0] * invNo; od.y += g1[1] * invNo; od.z += g1[2] * invNo; od.w += g1[3] * invNo;
      ob.x += g2[0] * invNo; ob.y += g2[1] * invNo; ob.z += g2[2] * invNo; ob.w += g2[3] * invNo;
      *reinterpret_cast<float4*>(gd + i) = od;
      *reinterpret_cast<float4*>(gb + i) = ob;
    }
  }
  double v = acc.value();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += red[k];
    part[blockIdx.x] = s;
  }
}

// R = invNo * sum of the per-CTA partials: 256 threads, each adds a strided subset in order, then
// a fixed shuffle tree and a fixed order over the warps (deterministic)
__global__ void __launch_bounds__(256) k_reg_final(const double* __restrict__ part, int nparts, double invNo,
                                                   double* __restrict__ out) {
  __shared__ double red[8];
  double v = 0.0;
  for (int k = threadIdx.x; k < nparts; k += blockDim.x) v += part[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    *out = s * invNo;
  }
}

// max |C| over the volume: per-CTA maxima, then one CTA (|C| >= 0, so float order = bit order)
__global__ void __launch_bounds__(256) k_absmax(const float* __restrict__ c, size_t n, float* __restrict__ part) {
  __shared__ float red[8];
  float m = 0.f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(c[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < 8; ++k) m = fmaxf(m, red[k]);
    part[blockIdx.x] = m;
  }
}

__global__ void __launch_bounds__(256) k_l1_weights(const float* __restrict__ c, size_t n,
                                                    const float* __restrict__ part, int nparts, float eps,
                                                    float* __restrict__ w) {
  __shared__ float mx;
  if (threadIdx.x == 0) {
    float m = 0.f;
    for (int k = 0; k < nparts; ++k) m = fmaxf(m, part[k]);
    mx = m;
  }
  __syncthreads();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    w[i] = mx / (fabsf(c[i]) + eps);
}

static unsigned reg_grid(size_t n) { return (unsigned)std::min<size_t>((n + 255) / 256, 152 * 8); }

int reg_parts(size_t n) { return (int)reg_grid(n); }

// rows of the regularizer kernel: at most reg_grid(n) CTAs (its partial-sum array), one row each
static unsigned reg_rows_grid(int Ly, int Lz, size_t n) {
  return (unsigned)std::min<size_t>((size_t)Ly * Lz, reg_grid(n));
}

cudaError_t launch_regularize(const float* d, const float* b, const float* wd, const float* wb, int Lz, int Ly, int Lx,
                              double ad, double ab, double gam, float* gd, float* gb, double* part, double* loss,
                              cudaStream_t s) {
  const size_t n = (size_t)Lz * Ly * Lx;
  const float invNo = (float)(1.0 / (double)n);
  auto al16 = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
  if (Lx % 4 == 0 && al16(d) && al16(b) && (!wd || al16(wd)) && (!wb || al16(wb)) && (!gd || (al16(gd) && al16(gb)))) {
    const unsigned grid = reg_grid(n);
    if (gam != 0.0)
      (k_regularize4<true><<<grid, 256, 0, s>>>(d, b, wd, wb, Lz, Ly, Lx, (float)ad, (float)ab, (float)gam, invNo, gd,
                                                gb, part), note_launch());
    else
      (k_regularize4<false><<<grid, 256, 0, s>>>(d, b, wd, wb, Lz, Ly, Lx, (float)ad, (float)ab, 0.f, invNo, gd, gb,
                                                 part), note_launch());
    if (loss) (k_reg_final<<<1, 256, 0, s>>>(part, (int)grid, 1.0 / (double)n, loss), note_launch());
    return cudaGetLastError();
  }
  const unsigned grid = reg_rows_grid(Ly, Lz, n);
  if (gam != 0.0)
    (k_regularize<true><<<grid, 256, 0, s>>>(d, b, wd, wb, Lz, Ly, Lx, (float)ad, (float)ab, (float)gam, invNo, gd,
                                             gb, part), note_launch());
  else
    (k_regularize<false><<<grid, 256, 0, s>>>(d, b, wd, wb, Lz, Ly, Lx, (float)ad, (float)ab, 0.f, invNo, gd, gb,
                                              part), note_launch());
  if (loss) (k_reg_final<<<1, 256, 0, s>>>(part, (int)grid, 1.0 / (double)n, loss), note_launch());
  return cudaGetLastError();
}

cudaError_t launch_l1_weights(const float* c, size_t n, float eps, float* part, float* w, cudaStream_t s) {
  const unsigned grid = reg_grid(n);
  (k_absmax<<<grid, 256, 0, s>>>(c, n, part), note_launch());
  (k_l1_weights<<<grid, 256, 0, s>>>(c, n, part, (int)grid, eps, w), note_launch());
  return cudaGetLastError();
}

}  // namespace adorym
