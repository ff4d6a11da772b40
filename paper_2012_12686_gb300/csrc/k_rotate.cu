// Transmission volume (Eq. ri_modulation), with the rotation of the object for ptychographic
// tomography (Eq. rotation_transform) fused in, and the rotation's exact transpose.  The plane perpendicular to the rotation axis (y) is the x-z plane; a rotated-frame
// voxel (z_t, y, x_t) samples the unrotated volume at
//   x0 = c (x_t - cx) - s (z_t - cz) + cx,   z0 = s (x_t - cx) + c (z_t - cz) + cz
// with bilinear weights; nodes outside the volume contribute nothing.  The transpose is computed
// in gather form (each unrotated node collects the rotated-frame voxels whose sample point lies
// within one pixel of it, with the forward pass's own weights), so it needs no atomics and is
// deterministic.
#include <algorithm>

#include "kernels.cuh"

namespace adorym {

struct Tap {
  int fx, fz;
  float ax, az;
};

__device__ __forceinline__ Tap tap(int zt, int xt, int Lz, int Lx, float c, float s) {
  const float cx = 0.5f * (float)(Lx - 1), cz = 0.5f * (float)(Lz - 1);
  const float u = (float)xt - cx, w = (float)zt - cz;
  const float x0 = fmaf(c, u, fmaf(-s, w, cx));
  const float z0 = fmaf(s, u, fmaf(c, w, cz));
  Tap t;
  const float fx = floorf(x0), fz = floorf(z0);
  t.fx = (int)fx;
  t.fz = (int)fz;
  t.ax = x0 - fx;
  t.az = z0 - fz;
  return t;
}

// T = exp(-kdz beta) exp(i kdz delta) of the (optionally rotated) volume, Eq. ri_modulation.
// Computed once per call so the fused kernel gathers a complex64 per voxel instead of
// evaluating sincos/exp for every (position, slice, pixel) it touches.
template <bool ROT>
__global__ void k_transmission(const float* __restrict__ vd, const float* __restrict__ vb, float2* __restrict__ T,
                               int Lz, int Ly, int Lx, float kdz, float c, float s) {
  const size_t n = (size_t)Lz * Ly * Lx;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float sd, sb;
    if (ROT) {
      const int xt = (int)(i % Lx);
      const int y = (int)((i / Lx) % Ly);
      const int zt = (int)(i / ((size_t)Lx * Ly));
      const Tap t = tap(zt, xt, Lz, Lx, c, s);
      sd = 0.f;
      sb = 0.f;
#pragma unroll
      for (int dz = 0; dz < 2; ++dz) {
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          const int z = t.fz + dz, x = t.fx + dx;
          if (z < 0 || z >= Lz || x < 0 || x >= Lx) continue;
          const float w = (dz ? t.az : 1.f - t.az) * (dx ? t.ax : 1.f - t.ax);
          const size_t o = ((size_t)z * Ly + y) * Lx + x;
          sd = fmaf(w, __ldg(vd + o), sd);
          sb = fmaf(w, __ldg(vb + o), sb);
        }
      }
    } else {
      sd = __ldg(vd + i);
      sb = __ldg(vb + i);
    }
    float sn, cs;
    sincosf(kdz * sd, &sn, &cs);
    const float e = expf(-kdz * sb);
    T[i] = make_float2(e * cs, e * sn);
  }
}

__global__ void k_rotate_adj(const double* __restrict__ gdr, const double* __restrict__ gbr, float* __restrict__ gd,
                             float* __restrict__ gb, int Lz, int Ly, int Lx, float c, float s) {
  const size_t n = (size_t)Lz * Ly * Lx;
  const float cx = 0.5f * (float)(Lx - 1), cz = 0.5f * (float)(Lz - 1);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % Lx);
    const int y = (int)((i / Lx) % Ly);
    const int z = (int)(i / ((size_t)Lx * Ly));
    // rotated-frame point that maps exactly onto this node (inverse rotation)
    const float u = (float)x - cx, w = (float)z - cz;
    const float xs = c * u + s * w + cx, zs = -s * u + c * w + cz;
    const int xa = max(0, (int)floorf(xs - 1.5f)), xb = min(Lx - 1, (int)ceilf(xs + 1.5f));
    const int za = max(0, (int)floorf(zs - 1.5f)), zb = min(Lz - 1, (int)ceilf(zs + 1.5f));
    double ad = 0.0, ab = 0.0;
    for (int zt = za; zt <= zb; ++zt) {
      for (int xt = xa; xt <= xb; ++xt) {
        const Tap t = tap(zt, xt, Lz, Lx, c, s);
        float wx, wz;
        if (t.fx == x) wx = 1.f - t.ax;
        else if (t.fx + 1 == x) wx = t.ax;
        else continue;
        if (t.fz == z) wz = 1.f - t.az;
        else if (t.fz + 1 == z) wz = t.az;
        else continue;
        const double wt = (double)(wx * wz);
        const size_t o = ((size_t)zt * Ly + y) * Lx + xt;
        ad = fma(wt, __ldg(gdr + o), ad);
        ab = fma(wt, __ldg(gbr + o), ab);
      }
    }
    gd[i] = (float)((double)gd[i] + ad);
    gb[i] = (float)((double)gb[i] + ab);
  }
}

cudaError_t launch_transmission(const float* vd, const float* vb, float2* T, int Lz, int Ly, int Lx, float kdz,
                                int rotate, float c, float sn, cudaStream_t s) {
  const size_t n = (size_t)Lz * Ly * Lx;
  const unsigned grid = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 16);
  if (rotate) k_transmission<true><<<grid, 256, 0, s>>>(vd, vb, T, Lz, Ly, Lx, kdz, c, sn);
  else k_transmission<false><<<grid, 256, 0, s>>>(vd, vb, T, Lz, Ly, Lx, kdz, c, sn);
  return cudaGetLastError();
}

cudaError_t launch_rotate_adj(const double* gdr, const double* gbr, float* gd, float* gb, int Lz, int Ly, int Lx,
                              float c, float sn, cudaStream_t s) {
  const size_t n = (size_t)Lz * Ly * Lx;
  const unsigned grid = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 16);
  k_rotate_adj<<<grid, 256, 0, s>>>(gdr, gbr, gd, gb, Lz, Ly, Lx, c, sn);
  return cudaGetLastError();
}

cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t s) { return cudaMemsetAsync(p, 0, bytes, s); }

__global__ void k_grad_add(const double* __restrict__ ad, const double* __restrict__ ab, float* __restrict__ gd,
                           float* __restrict__ gb, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    gd[i] = (float)((double)gd[i] + ad[i]);
    gb[i] = (float)((double)gb[i] + ab[i]);
  }
}

cudaError_t launch_grad_add(const double* ad, const double* ab, float* gd, float* gb, size_t n, cudaStream_t s) {
  const unsigned grid = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 16);
  k_grad_add<<<grid, 256, 0, s>>>(ad, ab, gd, gb, n);
  return cudaGetLastError();
}

}  // namespace adorym
