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
#include "numerics.cuh"

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

// Region of the volume a call touches: rows / columns covered by the batch's patches (far field)
// or the whole slab (near field), clamped to the volume, as box = {y0, y1, x0, x1}.  With
// full_x the column range is the whole width (tomography: the rotation transpose mixes x and z).
__global__ void __launch_bounds__(256) k_bbox(const float* __restrict__ pos, int B, int N, int Ly, int Lx, int far,
                                              int full_x, int* __restrict__ box, int npos_values,
                                              int* __restrict__ status, int* __restrict__ zero, int nzero) {
  __shared__ int red[4][8];
  for (int i = threadIdx.x; i < nzero; i += 256) zero[i] = 0;
  // input check: every position / shift value finite and within +-2^24 px
  bool bad = false;
  for (int i = threadIdx.x; i < npos_values; i += 256) {
    const float v = pos[i];
    bad |= !(fabsf(v) <= 16777216.f);   // also catches NaN
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) set_status(status, STATUS_BAD_POSITION);
  int y0 = 1 << 30, y1 = -(1 << 30), x0 = 1 << 30, x1 = -(1 << 30);
  if (far) {
    for (int b = threadIdx.x; b < B; b += 256) {
      const int py = patch_corner(pos[2 * b]), px = patch_corner(pos[2 * b + 1]);
      y0 = min(y0, py);
      y1 = max(y1, py + N);
      x0 = min(x0, px);
      x1 = max(x1, px + N);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    y0 = min(y0, __shfl_xor_sync(0xffffffffu, y0, o));
    y1 = max(y1, __shfl_xor_sync(0xffffffffu, y1, o));
    x0 = min(x0, __shfl_xor_sync(0xffffffffu, x0, o));
    x1 = max(x1, __shfl_xor_sync(0xffffffffu, x1, o));
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = y0;
    red[1][w] = y1;
    red[2][w] = x0;
    red[3][w] = x1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < 8; ++i) {
      y0 = min(y0, red[0][i]);
      y1 = max(y1, red[1][i]);
      x0 = min(x0, red[2][i]);
      x1 = max(x1, red[3][i]);
    }
    if (!far) {
      y0 = 0;
      y1 = Ly;
      x0 = 0;
      x1 = Lx;
    }
    box[0] = max(0, y0);
    box[1] = min(Ly, y1);
    box[2] = full_x ? 0 : max(0, x0);
    box[3] = full_x ? Lx : min(Lx, x1);
  }
}

struct Region {
  int y0, h, x0, w;
  size_t n;   // Lz * h * w
};

__device__ __forceinline__ Region region(const int* __restrict__ box, int Lz) {
  Region r;
  r.y0 = box[0];
  r.h = max(0, box[1] - box[0]);
  r.x0 = box[2];
  r.w = max(0, box[3] - box[2]);
  r.n = (size_t)Lz * r.h * r.w;
  return r;
}

// Work split of the box kernels below: a warp takes one chunk of PER_LANE x 32 consecutive voxels
// of a box row (z, y) at a time, lanes along x, so the row and column of a voxel come from one
// integer division per chunk instead of per voxel, and each lane keeps PER_LANE loads in flight.
struct BoxChunks {
  static constexpr int PER_LANE = 4;
  unsigned y0, h, cpr, items;   // first box row, box rows per slice, chunks per row, chunks in the box
  __device__ BoxChunks(const Region& R, int Lz) {
    y0 = (unsigned)R.y0;
    h = (unsigned)R.h;
    cpr = (unsigned)((R.w + 32 * PER_LANE - 1) / (32 * PER_LANE));
    items = (unsigned)Lz * h * cpr;
  }
  __device__ static unsigned first() { return (blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
  __device__ static unsigned stride() { return (gridDim.x * blockDim.x) >> 5; }
  // chunk -> slice z, volume row y, first column xc of the chunk relative to the box
  __device__ void split(unsigned item, int* z, int* y, int* xc) const {
    const unsigned row = item / cpr, c = item - row * cpr;
    const unsigned zz = row / h;
    *z = (int)zz;
    *y = (int)(y0 + row - zz * h);
    *xc = (int)c * 32 * PER_LANE;
  }
};

// T = exp(-kdz beta) exp(i kdz delta) of the (optionally rotated) volume over the box, Eq.
// ri_modulation.  Computed once per call so the fused kernels gather a complex64 per voxel
// instead of evaluating sincos/exp for every (position, slice, pixel) they touch.
template <bool ROT>
__global__ void __launch_bounds__(256) k_transmission(const float* __restrict__ vd, const float* __restrict__ vb,
                                                      float2* __restrict__ T, int Lz, int Ly, int Lx, float kdz,
                                                      float c, float s, const int* __restrict__ box,
                                                      double* __restrict__ zero_a, double* __restrict__ zero_b) {
  const Region R = region(box, Lz);
  BoxChunks K(R, Lz);
  constexpr int U = BoxChunks::PER_LANE;
  for (unsigned item = K.first(); item < K.items; item += K.stride()) {
    int zt, y, xc;
    K.split(item, &zt, &y, &xc);
    const size_t base = ((size_t)zt * Ly + y) * Lx;
    const int x0 = xc + (int)(threadIdx.x & 31);
    // all of the chunk's loads first, so that they are in flight together: one voxel per lane
    // and step u (unrotated volume), or the four bilinear taps of each (rotated volume)
    float ld[U][ROT ? 4 : 1], lb[U][ROT ? 4 : 1];
    Tap tp[ROT ? U : 1];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int xi = x0 + 32 * u;
      const bool in = xi < R.w;
      if (ROT) {
        tp[ROT ? u : 0] = tap(zt, R.x0 + xi, Lz, Lx, c, s);
        const Tap& t = tp[ROT ? u : 0];
#pragma unroll
        for (int q = 0; q < (ROT ? 4 : 1); ++q) {
          const int z = t.fz + (q >> 1), x = t.fx + (q & 1);
          const bool ok = in && z >= 0 && z < Lz && x >= 0 && x < Lx;
          const size_t o = ((size_t)z * Ly + y) * Lx + x;
          ld[u][q] = ok ? __ldg(vd + o) : 0.f;
          lb[u][q] = ok ? __ldg(vb + o) : 0.f;
        }
      } else {
        ld[u][0] = in ? __ldg(vd + base + R.x0 + xi) : 0.f;
        lb[u][0] = in ? __ldg(vb + base + R.x0 + xi) : 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int xi = x0 + 32 * u;
      if (xi >= R.w) break;
      const int xt = R.x0 + xi;
      const size_t io = base + xt;
      float sd, sb;
      if (ROT) {
        // taps in (dz, dx) order, those outside the volume skipped
        const Tap& t = tp[ROT ? u : 0];
        sd = 0.f;
        sb = 0.f;
#pragma unroll
        for (int q = 0; q < (ROT ? 4 : 1); ++q) {
          const int dz = q >> 1, dx = q & 1, z = t.fz + dz, x = t.fx + dx;
          if (z < 0 || z >= Lz || x < 0 || x >= Lx) continue;
          const float w = (dz ? t.az : 1.f - t.az) * (dx ? t.ax : 1.f - t.ax);
          sd = fmaf(w, ld[u][q], sd);
          sb = fmaf(w, lb[u][q], sb);
        }
      } else {
        sd = ld[u][0];
        sb = lb[u][0];
      }
      float sn, cs;
      sincosf(kdz * sd, &sn, &cs);
      const float e = expf(-kdz * sb);
      T[io] = make_float2(e * cs, e * sn);
      if (zero_a) {
        zero_a[io] = 0.0;
        zero_b[io] = 0.0;
      }
    }
  }
}

// transpose of the rotation, step 1 (per call, independent of y): for each unrotated node (z, x)
// the rotated-frame nodes (z_t, x_t) whose sample point lies within one pixel of it, with the
// forward pass's own bilinear weights, in the order z_t, then x_t ascending.  Table planes of
// P = Lz * Lx ints: [0] count, [1 + k] packed node z_t * 65536 + x_t, [1 + kRotTaps + k] weight.
__global__ void __launch_bounds__(256) k_rotate_table(int* __restrict__ tab, int Lz, int Lx, float c, float s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int P = Lz * Lx;
  if (i >= P) return;
  const int z = i / Lx, x = i - z * Lx;
  const float cx = 0.5f * (float)(Lx - 1), cz = 0.5f * (float)(Lz - 1);
  // rotated-frame point that maps exactly onto this node (inverse rotation)
  const float u = (float)x - cx, w = (float)z - cz;
  const float xs = c * u + s * w + cx, zs = -s * u + c * w + cz;
  // a contributing voxel samples within one pixel of the node in x and z, so (inverse rotation)
  // it lies within |c| + |s| <= sqrt(2) of (xs, zs) along each axis: at most 3 x 3 candidates
  // (the margin covers FP32 rounding of xs, zs and of the forward taps); the membership test
  // below is the forward pass's own
  const float r = fabsf(c) + fabsf(s) + 0.01f;
  const int xa = max(0, (int)ceilf(xs - r)), xb = min(Lx - 1, (int)floorf(xs + r));
  const int za = max(0, (int)ceilf(zs - r)), zb = min(Lz - 1, (int)floorf(zs + r));
  int n = 0;
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
      if (n < kRotTaps) {   // always true: at most 3 x 3 candidates
        tab[(size_t)(1 + n) * P + i] = (zt << 16) | xt;
        tab[(size_t)(1 + kRotTaps + n) * P + i] = __float_as_int(wx * wz);
        ++n;
      }
    }
  }
  tab[i] = n;
}

// step 2: each unrotated node (z, y, x) of the box collects its rotated-frame accumulators from
// the table (flat index over the box's rows and columns, threads along x).  The taps are FP64
// sums over positions; each is narrowed once (integer arithmetic, round to nearest) and the
// weighted taps are added in FP32 in the table's order, like the caller's FP32 gradient
__global__ void __launch_bounds__(256) k_rotate_adj(const double* __restrict__ gdr, const double* __restrict__ gbr,
                                                    float* __restrict__ gd, float* __restrict__ gb, int Lz, int Ly,
                                                    int Lx, const int* __restrict__ tab, const int* __restrict__ box) {
  const Region R = region(box, Lz);
  const int P = Lz * Lx;
  const unsigned n = (unsigned)R.n;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned row = i / (unsigned)R.w;
    const int x = R.x0 + (int)(i - row * (unsigned)R.w);
    const int z = (int)(row / (unsigned)R.h), y = R.y0 + (int)(row - (unsigned)z * (unsigned)R.h);
    const int node = z * Lx + x;
    const int cnt = __ldg(tab + node);
    float ad = 0.f, ab = 0.f;
    for (int k = 0; k < cnt; ++k) {
      const int zx = __ldg(tab + (size_t)(1 + k) * P + node);
      const float wk = __int_as_float(__ldg(tab + (size_t)(1 + kRotTaps + k) * P + node));
      const size_t o = ((size_t)(zx >> 16) * Ly + y) * Lx + (zx & 0xFFFF);
      ad = fmaf(wk, f64_to_f32(gdr + o), ad);
      ab = fmaf(wk, f64_to_f32(gbr + o), ab);
    }
    const size_t io = ((size_t)z * Ly + y) * Lx + x;
    gd[io] += ad;
    gb[io] += ab;
  }
}

// FP64 object-gradient accumulators (zeroed over the box by the transmission pass): add the box
// into the caller's gradient (work split as in BoxChunks)
__global__ void __launch_bounds__(256) k_grad_add(const double* __restrict__ ad, const double* __restrict__ ab,
                                                  float* __restrict__ gd, float* __restrict__ gb, int Lz, int Ly,
                                                  int Lx, const int* __restrict__ box) {
  const Region R = region(box, Lz);
  BoxChunks K(R, Lz);
  constexpr int U = BoxChunks::PER_LANE;
  for (unsigned item = K.first(); item < K.items; item += K.stride()) {
    int z, y, xc;
    K.split(item, &z, &y, &xc);
    const size_t base = ((size_t)z * Ly + y) * Lx + R.x0;
    const int x0 = xc + (int)(threadIdx.x & 31);
    // all of the chunk's loads first (in flight together), then the adds and stores
    float gd_[U], gb_[U], ad_[U], ab_[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool in = x0 + 32 * u < R.w;
      const size_t io = base + x0 + 32 * u;
      ad_[u] = in ? f64_to_f32(ad + io) : 0.f;   // narrowed in integer arithmetic
      ab_[u] = in ? f64_to_f32(ab + io) : 0.f;
      gd_[u] = in ? gd[io] : 0.f;
      gb_[u] = in ? gb[io] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (x0 + 32 * u >= R.w) break;
      const size_t io = base + x0 + 32 * u;
      gd[io] = gd_[u] + ad_[u];   // one FP32 add
      gb[io] = gb_[u] + ab_[u];
    }
  }
}

static unsigned vol_grid(size_t n) { return (unsigned)std::min<size_t>((n + 255) / 256, 152 * 16); }
// one warp per BoxChunks chunk of a box inside Lz x Ly x Lx (eight warps per block), at most 16
// blocks per SM; the warps loop over the chunks beyond that
static unsigned box_grid(int Lz, int Ly, int Lx) {
  const size_t chunks = (size_t)Lz * Ly * (((size_t)Lx + 127) / 128);
  return (unsigned)std::min<size_t>((chunks + 7) / 8, 152 * 16);
}

cudaError_t launch_bbox(const float* pos, int B, int N, int Ly, int Lx, int far, int full_x, int* box,
                        int npos_values, int* status, cudaStream_t s, int* zero, int nzero) {
  (k_bbox<<<1, 256, 0, s>>>(pos, B, N, Ly, Lx, far, full_x, box, npos_values, status, zero, nzero), note_launch());
  return cudaGetLastError();
}

cudaError_t launch_transmission(const float* vd, const float* vb, float2* T, int Lz, int Ly, int Lx, float kdz,
                                int rotate, float c, float sn, const int* box, double* zero_a, double* zero_b,
                                cudaStream_t s) {
  const unsigned grid = box_grid(Lz, Ly, Lx);
  if (rotate) (k_transmission<true><<<grid, 256, 0, s>>>(vd, vb, T, Lz, Ly, Lx, kdz, c, sn, box, zero_a, zero_b), note_launch());
  else (k_transmission<false><<<grid, 256, 0, s>>>(vd, vb, T, Lz, Ly, Lx, kdz, c, sn, box, zero_a, zero_b), note_launch());
  return cudaGetLastError();
}

cudaError_t launch_rotate_adj(const double* gdr, const double* gbr, float* gd, float* gb, int Lz, int Ly, int Lx,
                              float c, float sn, const int* box, int* tab, cudaStream_t s) {
  const int nodes = Lz * Lx;
  (k_rotate_table<<<(nodes + 255) / 256, 256, 0, s>>>(tab, Lz, Lx, c, sn), note_launch());
  (k_rotate_adj<<<vol_grid((size_t)Lz * Ly * Lx), 256, 0, s>>>(gdr, gbr, gd, gb, Lz, Ly, Lx, tab, box), note_launch());
  return cudaGetLastError();
}

cudaError_t launch_grad_add(const double* ad, const double* ab, float* gd, float* gb, int Lz, int Ly, int Lx,
                            const int* box, cudaStream_t s) {
  (k_grad_add<<<box_grid(Lz, Ly, Lx), 256, 0, s>>>(ad, ab, gd, gb, Lz, Ly, Lx, box), note_launch());
  return cudaGetLastError();
}

cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t s) { return cudaMemsetAsync(p, 0, bytes, s); }

}  // namespace adorym
