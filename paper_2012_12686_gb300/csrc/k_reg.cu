// Regularizers of Table regularizers in the refractive-index form, added to the data term as in
// Eq. tikhonov:
//   R = (1/N_o) [ sum a_d W_d |delta| + a_b W_b |beta| + gamma sum_axes (|grad delta| + |grad beta|) ]
// with forward differences (no term past the last index), subgradient 0 at 0, and optional
// reweighting W = max|C| / (|C| + eps) from a snapshot.  Dense volume work, HBM-bound: one pass
// reads delta, beta (and W), each voxel gathers its own TV subgradient from its neighbours (no
// atomics), per-CTA FP64 partial sums are added in a fixed order.
#include <algorithm>

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

__global__ void k_reg_final(const double* __restrict__ part, int nparts, double invNo, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < nparts; ++k) s += part[k];
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
  const unsigned grid = reg_rows_grid(Ly, Lz, n);
  const float invNo = (float)(1.0 / (double)n);
  if (gam != 0.0)
    (k_regularize<true><<<grid, 256, 0, s>>>(d, b, wd, wb, Lz, Ly, Lx, (float)ad, (float)ab, (float)gam, invNo, gd,
                                             gb, part), note_launch());
  else
    (k_regularize<false><<<grid, 256, 0, s>>>(d, b, wd, wb, Lz, Ly, Lx, (float)ad, (float)ab, 0.f, invNo, gd, gb,
                                              part), note_launch());
  if (loss) (k_reg_final<<<1, 32, 0, s>>>(part, (int)grid, 1.0 / (double)n, loss), note_launch());
  return cudaGetLastError();
}

cudaError_t launch_l1_weights(const float* c, size_t n, float eps, float* part, float* w, cudaStream_t s) {
  const unsigned grid = reg_grid(n);
  (k_absmax<<<grid, 256, 0, s>>>(c, n, part), note_launch());
  (k_l1_weights<<<grid, 256, 0, s>>>(c, n, part, (int)grid, eps, w), note_launch());
  return cudaGetLastError();
}

}  // namespace adorym
