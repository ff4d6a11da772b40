// Device-side argument blocks and host launchers shared by the kernel files and the C ABI.
#pragma once
#include <cuda.h>   // CUtensorMap (type only; encoded through the runtime's driver entry point)
#include <cuda_runtime.h>
#include <atomic>
#include <cstddef>
#include <cstdint>

namespace adorym {

// Kernels launched (or recorded into a captured graph) by this library in this process; every
// launch site adds one (adorym_kernel_launches reports it)
extern std::atomic<unsigned long long> g_kernel_launches;
inline void note_launch() { g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }

// kernel attributes are per device: the "already prepared" caches are indexed by the current
// device (up to this many) and atomic, as several contexts may prepare from different threads
constexpr int kMaxDevices = 64;
inline int current_device() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return (d >= 0 && d < kMaxDevices) ? d : -1;
}

// One far-field (or near-field) loss/gradient launch over a batch, as seen by the fused kernel.
struct PathArgs {
  int N, L, M, B, Ly, Lx;
  int cp, ncp;            // checkpoint spacing and count (ncp = ceil(L / cp))
  int loss;               // 0 = LSQ (Eq. lsq_loss), 1 = Poisson (Eq. poisson_loss)
  int adj;                // 1: run the adjoint (loss_grad); 0: forward only
  int n_dist;             // near field: number of sample-detector distances
  int pipe;               // 1: two-CTA clusters per position (grid 2 B); seg holds two slot sets
  float eps, kdz;
  double inv_npix;        // 1 / (number of detector pixels in the batch)
  const float2* T;        // transmission exp(i kdz (delta + i beta)) [Lz][Ly][Lx] (rotated frame for tomography)
  const float2* probe;    // near field: illumination [M][N][N]
  const float2* phat;     // far field: DFT_-[probe] [M][N][N]
  const float* pos;       // far field [B][2] (y, x); near field shifts [B][n_dist][2]
  const float* I_meas;    // [B][N][N] or [B][n_dist][N][N]; null for forward-only
  float* I_out;           // predicted intensities (same shape) or null
  const float2* tw;       // W_N^m = exp(-2 pi i m / N), m < N
  const float2* hy;       // slice-to-slice propagator factors exp(i pi c f^2) / N
  const float2* hx;
  const float2* hd;       // near field: [n_dist][N] factors exp(i pi f^2 / N_F) (unscaled)
  float2* ckpt;           // [B][M][ncp][N*N] checkpoints psi_{j0}
  float2* seg;            // [B][M][cp][N*N] recomputed psi_j of one segment
  float2* park;           // [B][N*(N+1)] adjoint field parked during a recompute
  float2* far;            // [B][M][N*N] detector field (far) or [B][n_dist][M][N*N] (near)
  float* gI;              // [B][N*N] (or [B][n_dist][N*N]) intensity, then dL/dI
  float2* fbar;           // near field: [B][N*N] accumulated Fourier-space adjoint
  double* lossp;          // [B] per-problem loss sums
  float2* qacc;           // [B][M][N*N] per-position probe-gradient partials (Fourier space)
  double* gd;             // FP64 object-gradient accumulator [Lz][Ly][Lx] (+=), or null
  double* gb;
  // near field with one probe mode: every voxel receives exactly one term per call, so it is
  // added straight into the caller's FP32 gradient (no accumulator, no atomics); else null
  float* gdf;
  float* gbf;
  float* gpos;            // [B][2] or [B][n_dist][2] (overwritten), or null
  double* gposd;          // far field: [B][2] the same position gradients in FP64 (for the
                          // per-angle offset sum), or null
  float* gnf;             // near field: [B][n_dist] dL/dN_F (overwritten), or null
  double nf[4];           // near field: Fresnel numbers
  // sparse / variable multislice: per-gap propagator factors [L-1][N] (null: uniform hy, hx)
  const float2* hyj;
  const float2* hxj;
  // recompute helpers (uniform spacing, one CTA per position, batch below the SM count): CTAs
  // blockIdx.x >= B recompute segments 0..ncp-2 into hseg while the positions run; the control
  // words are zeroed by the bounding-box kernel before each launch
  int helpers;            // helper CTAs (grid B + helpers); 0: none
  float2* hseg;           // [B][M][ncp-1][cp][N*N] helper-recomputed psi_j (slice 0 of a segment unused)
  int* hnext;             // next helper task (segment-major: s, then m, then b)
  int* hprog;             // [B][M] checkpoints the forward has written so far (release / acquire)
  int* hflag;             // [B][M][ncp] 0 free, 1 helper recomputing, 2 helper done, 3 taken by the position
  float2* spck;           // gap gradient: spectra F[psi_j] / N^2 of checkpoint slices [B][M][ncp][N*N]
  float2* spseg;          //               and of segment slices [B][M][cp][N*N]
  double* gapp;           // [B][L-1] per-position slice-gap gradient partials, or null
  long long wait_seg;     // cycle limits of the helper protocol's waits (a position for a helper's
  long long wait_ckpt;    // segment; a helper for a checkpoint): WaitLimits
};

// Arguments of the two-pass path (N >= 256): fields in HBM, one row and one column kernel per
// slice step.  The per-launch fields (m, j, s, j0, j1, d, buf) select the step.
struct TPArgs {
  int N, L, M, B, Ly, Lx, cp, ncp, nd, loss, farfield, adj;
  float eps, kdz;
  double inv_npix;
  const float2* T;         // transmission volume [Lz][Ly][Lx]
  const float2* probe;     // [M][N][N]
  const float2* phat;      // [M][N][N] DFT_-[probe] (natural frequency order)
  float2* phat_w;          // same buffer, written by the probe transform
  const float* pos;
  const float* I_meas;
  float* I_out;
  const float2* tw;
  const float2* hy;        // exp(i pi c f^2) / N
  const float2* hx;
  const float2* hd;        // near field [n_dist][N] exp(i pi f^2 / N_F)
  float2* FA;              // [B][M][N*N] forward / adjoint field
  float2* FR;              // [B][M][N*N] recompute field
  float2* ckpt;            // [B][M][ncp][N*N]
  float2* seg;             // [B][M][cp][N*N]
  float2* far;             // far [B][M][N*N]; near [B][n_dist + 1][M][N*N] (Psi_d, then Phi)
  float* gI;               // [B][n_dist][N*N]
  double* lossp;           // [B * n_dist][N*N / 1024] loss partials
  double* posp;            // [B][n_dist][N / CW][3] shift (y, x) and Fresnel-number gradient partials
  float2* qacc;            // [B][M][N*N]
  float2* qsum;            // [M][N*N]
  float2* tmp;             // [M][N*N]
  double* gd;              // FP64 object-gradient accumulator
  double* gb;
  float* gdf;              // direct FP32 object gradient (near field, one probe mode), else null
  float* gbf;
  float* gpos;
  double* gposd;           // far field: [B][2] position gradients in FP64, or null
  float* gnf;
  double nf[4];
  const float2* hyj;       // variable slice spacing: per-gap propagator factors [L-1][N], or null
  const float2* hxj;
  float2* spec_out;        // per launch: base of the spectra array to write [B][M][spo_n][N*N] (or null)
  const float2* spec_in;   // per launch: base of the spectra array to read  [B][M][spi_n][N*N] (or null)
  int spo_slot, spo_n, spi_slot, spi_n;
  double* gapp;            // [B][L-1][N / CW] slice-gap gradient partials, or null
  float* ggap;             // [L-1] output
  float2* g_probe;
  double* loss_out;
  int* status;             // the call's device status word (STATUS_* bits)
  // TMA staging of the column kernels' tiles: 2-D maps over the field buffers FA, FR, far, tmp
  // (rows of N complex64, box CW x min(N, 256)); tma = 0 falls back to register-staged loads
  int tma;
  unsigned long long tm_rows[4];
  CUtensorMap tm[4];
  int m, j, s, j0, j1, d, buf;
  long long wait_tma;      // cycle limit of a column tile's TMA wait (negative: report a timeout at once)
};

// Cycle limits of the bounded device-side waits, read by every later call when it is enqueued
// (adorym_set_wait_limits changes them for tests of the fallback branches)
struct WaitLimits {
  long long seg = 1LL << 28;    // a position waiting for a segment a helper is recomputing
  long long ckpt = 1LL << 24;   // a helper waiting for a position's checkpoint
  long long tma = 1LL << 31;    // a column tile's TMA copy
};
WaitLimits wait_limits();

// launchers (return cudaGetLastError())
cudaError_t launch_probe_hat(int N, int M, const float2* probe, float2* phat, const float2* tw, cudaStream_t s);
cudaError_t launch_path(const PathArgs& a, int farfield, cudaStream_t s);
// the variable-spacing instantiation (a.hyj != nullptr), compiled in its own translation unit
cudaError_t launch_path_gaps(const PathArgs& a, int farfield, cudaStream_t s);
cudaError_t prepare_path_gaps(int N, int farfield);
// the pipelined two-CTA-cluster instantiation (a.pipe != 0), in its own translation unit
cudaError_t launch_path_pipe(const PathArgs& a, int farfield, cudaStream_t s);
cudaError_t prepare_path_pipe(int N, int farfield);
// the instantiation with recompute helpers (a.helpers > 0), in its own translation unit
cudaError_t launch_path_help(const PathArgs& a, int farfield, cudaStream_t s);
cudaError_t prepare_path_help(int N, int farfield);
// per-angle position offset (Sec. 2.3.2): g_off[a] = sum_b gposd[b][a] in FP64, fixed order
cudaError_t launch_offset_sum(const double* gposd, int B, float* g_off, cudaStream_t s);
// g_gap[j] = sum_b gapp[b][j][k] over b and k < parts (fixed order)
cudaError_t launch_gap_final(const double* gapp, int B, int ngap, int parts, float* g_gap, cudaStream_t s);
cudaError_t launch_probe_grad(int N, int M, int B, int farfield, const float2* qacc, float2* qsum, float2* g_probe,
                              const float2* tw, const double* lossp, double inv_npix, double* loss_out,
                              cudaStream_t s);
// box = {y0, y1, x0, x1}: rows / columns of the volume the batch's patches touch (whole width if
// full_x), computed on the device from the positions
// status word bits set by the kernels (the host maps any bit to ADORYM_EDATA)
constexpr int STATUS_BAD_POSITION = 1;   // a position / shift is not finite or beyond +-2^24 px
constexpr int STATUS_WAIT_TIMEOUT = 2;   // a bounded device-side wait (TMA completion) gave up
// npos_values: 2 B (far field) or 2 B n_dist (near-field shifts) floats checked into *status
// also zeroes nzero ints at zero (the fused kernel's helper control words), when given
cudaError_t launch_bbox(const float* pos, int B, int N, int Ly, int Lx, int far, int full_x, int* box,
                        int npos_values, int* status, cudaStream_t s, int* zero = nullptr, int nzero = 0);
// T = exp(-kdz beta) exp(i kdz delta) over the box (Eq. ri_modulation), optionally after the
// bilinear rotation of Eq. rotation_transform (rotate = 1); zero_a / zero_b (FP64 object-gradient
// accumulators over the same box) are zeroed in the same pass when non-null
cudaError_t launch_transmission(const float* vd, const float* vb, float2* T, int Lz, int Ly, int Lx, float kdz,
                                int rotate, float c, float sn, const int* box, double* zero_a, double* zero_b,
                                cudaStream_t s);
// The rotation's transpose per unrotated node (z, x), independent of y: the rotated-frame nodes
// (z_t, x_t) that contribute and their bilinear weights.  The candidates lie in a 3 x 3 window
// (|cos| + |sin| <= sqrt 2 on each side), so nine entries always suffice (up to five contribute
// at some angles).  Stored as planes over the Lz * Lx nodes (coalesced reads): a count, then per
// entry k the packed node z_t * 65536 + x_t and the weight.
constexpr int kRotTaps = 9;
inline size_t rot_table_ints(int Lz, int Lx) { return (size_t)Lz * Lx * (1 + 2 * kRotTaps); }
// transpose of the rotation applied to the FP64 rotated-frame accumulators, added into gd/gb (rows
// of the box); tab: rot_table_ints(Lz, Lx) ints of scratch, filled by the call (Lz, Lx < 65536)
cudaError_t launch_rotate_adj(const double* gd_rot, const double* gb_rot, float* gd, float* gb, int Lz, int Ly,
                              int Lx, float c, float sn, const int* box, int* tab, cudaStream_t s);
// FP64 accumulators: add the box into the caller's FP32 gradient
cudaError_t launch_grad_add(const double* acc_d, const double* acc_b, float* gd, float* gb, int Lz, int Ly, int Lx,
                            const int* box, cudaStream_t s);
cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t s);
// regularizers (l1 / reweighted l1 / TV): part needs reg_parts(n) doubles
int reg_parts(size_t n);
cudaError_t launch_regularize(const float* d, const float* b, const float* wd, const float* wb, int Lz, int Ly, int Lx,
                              double ad, double ab, double gam, float* gd, float* gb, double* part, double* loss,
                              cudaStream_t s);
// W = max|C| / (|C| + eps); part needs reg_parts(n) floats
cudaError_t launch_l1_weights(const float* c, size_t n, float eps, float* part, float* w, cudaStream_t s);
// qsum[i] = sum_b qacc[b][i] in FP64, fixed order
cudaError_t launch_qsum(const float2* qacc, float2* qsum, int B, size_t MNN, cudaStream_t s);
int path_smem_bytes(int N);
// whole two-pass loss/gradient (adj = 1) or forward (adj = 0) sequence for N in {256, 512, 1024}
// meas_ready (or null): event of the measured intensities' copy; the stream waits for it just
// before the first kernel that reads them, so the copy overlaps the forward passes.  Near field
// with n_meas_part = n_dist: meas_part[d] marks distance d's intensities, and each detector pass
// waits only for its own distance
cudaError_t launch_twopass(TPArgs a, cudaStream_t s, cudaEvent_t ev_start, cudaEvent_t ev_stop,
                           cudaEvent_t meas_ready = nullptr, const cudaEvent_t* meas_part = nullptr,
                           int n_meas_part = 0);
cudaError_t prepare_twopass(int N);
// set the dynamic shared-memory attributes of every kernel used for tile size N (call outside capture)
cudaError_t prepare_path(int N, int farfield);

}  // namespace adorym
