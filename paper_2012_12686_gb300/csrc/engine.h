// Host-side engine shared by the direct C ABI entry points and the serving loop.
#pragma once
#include <cuda_runtime.h>

#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/adorym.h"
#include "kernels.cuh"

namespace adorym {

struct Object {
  const float* d = nullptr;
  const float* b = nullptr;
  int Lz = 0, Ly = 0, Lx = 0;
};

// Workspace layout of one call (byte offsets into one device allocation, 256-byte aligned).
struct Plan {
  adorym_problem p{};
  int cp = 1, ncp = 1, nd = 1;
  bool far = true, tomo = false, adj = false;
  bool want_obj = false, want_probe = false, want_pos = false, want_loss = false, want_nf = false;
  bool gaps = false, want_gaps = false;   // variable slice spacing / its gradient
  bool want_offset = false;                // far field: per-angle position offset gradient
  bool pipe = false;   // shared-memory path: two-CTA clusters (adjoint + segment recompute)
  int helpers = 0;     // shared-memory path: recompute-helper CTAs on SMs the batch leaves idle
  size_t NN = 0;
  size_t off_phat = 0, off_ckpt = 0, off_seg = 0, off_park = 0, off_far = 0, off_gI = 0, off_fbar = 0,
         off_lossp = 0, off_qacc = 0, off_qsum = 0, off_T = 0, off_grot = 0, off_loss = 0;
  // two-pass path (N >= 256)
  size_t off_FA = 0, off_FR = 0, off_tmp = 0, off_posp = 0;
  size_t off_box = 0;   // int4 bounding box of the batch's patches
  size_t off_hseg = 0, off_hctl = 0;   // helper segment store; helper control words (hnext, hprog, hflag)
  size_t off_status = 0;   // int device status word of the call (ADORYM_STATUS_* bits)
  size_t off_spck = 0, off_spseg = 0, off_gapp = 0, off_s_ggap = 0;   // slice-gap gradient
  size_t off_posd = 0, off_s_goff = 0;   // FP64 position gradients [B][2]; staged offset gradient
  size_t off_rtab = 0;                   // tomography: rotation-transpose table [Lz][Lx]
  // staging for host-memory arguments
  size_t off_s_probe = 0, off_s_pos = 0, off_s_meas = 0, off_s_gprobe = 0, off_s_gpos = 0, off_s_iout = 0,
         off_s_gnf = 0;
  size_t bytes_probe = 0, bytes_pos = 0, bytes_meas = 0, bytes_iout = 0;
  size_t total = 0;
};

// Device pointers of one call after staging.
struct CallPtrs {
  const float2* probe = nullptr;
  const float* pos = nullptr;
  const float* I_meas = nullptr;
  double* loss = nullptr;
  float* gd = nullptr;
  float* gb = nullptr;
  float2* g_probe = nullptr;
  float* g_pos = nullptr;
  float* g_nf = nullptr;
  float* I_out = nullptr;
  float* g_gaps = nullptr;
  float* g_offset = nullptr;   // far field: [2] per-angle position offset gradient (overwritten)
  // the measured intensities arrive on a side stream: the stream waits for this event before the
  // first kernel that reads them (the kernels before it overlap the copy); null when there is
  // nothing to wait for
  cudaEvent_t meas_ready = nullptr;
  // near field, two-pass path: the intensities of distance d arrive separately (meas_part[d],
  // n_meas_part = n_dist; meas_ready is then the last part), so each detector pass waits only
  // for its own distance
  const cudaEvent_t* meas_part = nullptr;
  int n_meas_part = 0;
  // shared-memory path: a second stream for the single-CTA probe kernels, forked from the call's
  // stream and joined back with ev_side = {fork 1, join 1, fork 2, join 2}: the probe transform
  // runs beside the bounding-box and transmission passes, the probe-gradient reduction and
  // transform beside the object-gradient pass.  Null: everything on the call's stream.
  cudaStream_t side = nullptr;
  cudaEvent_t ev_side[4] = {nullptr, nullptr, nullptr, nullptr};
  // device-visible status word to use instead of the plan's (not cleared by the call: the owner
  // zeroes it before the work runs); null: the workspace word, cleared on the stream
  int* status = nullptr;
};

int validate(const adorym_problem& p, const char** err);
bool two_pass(int N);   // N >= 256: fields in HBM, row/column kernels per slice step
int make_plan(const adorym_problem& p, bool adj, int grads, bool want_loss, Plan* plan, const char** err);
// direct calls on an otherwise idle device: give the fused kernel recompute helpers on the SMs a
// batch below the SM count leaves idle (extends the workspace; serving does not use them)
void plan_helpers(Plan* plan);
size_t helper_ctl_ints(const Plan& plan);
// FP64-built tables (twiddles, propagator factors) of a problem: table_count(p) float2 values
size_t table_count(const adorym_problem& p);
void fill_tables(const adorym_problem& p, float2* out);

struct Tables {
  float2* dev = nullptr;   // [tw N][hy N][hx N][hd n_dist*N][hyj (L-1)*N][hxj (L-1)*N]
  int N = 0, nd = 0, ngap = 0;
  const float2* tw() const { return dev; }
  const float2* hy() const { return dev + N; }
  const float2* hx() const { return dev + 2 * N; }
  const float2* hd() const { return dev + 3 * N; }
  const float2* hyj() const { return ngap ? dev + (size_t)(3 + nd) * N : nullptr; }
  const float2* hxj() const { return ngap ? dev + (size_t)(3 + nd) * N + (size_t)ngap * N : nullptr; }
};

// Enqueue every kernel of one call on `s` with workspace `ws` (no allocation, no host sync):
// safe inside CUDA stream capture.
int enqueue(const Plan& pl, const Object& obj, const Tables& tab, const CallPtrs& c, char* ws, cudaStream_t s,
            std::string* err, cudaEvent_t ev_start = nullptr, cudaEvent_t ev_stop = nullptr);

struct Serve;

}  // namespace adorym

struct adorym_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::mutex mu;                    // guards everything below
  std::string err;
  std::map<int, adorym::Object> objects;
  int next_obj = 1;
  char* ws = nullptr;
  size_t ws_cap = 0;
  std::map<std::string, adorym::Tables> tables;
  bool timing = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;   // fused-kernel timing pair
  cudaStream_t copy_stream = nullptr;          // host-to-device copy of measured intensities
  cudaEvent_t ev_fork = nullptr, ev_meas = nullptr;
  cudaEvent_t ev_meas_d[4] = {nullptr, nullptr, nullptr, nullptr};   // per-distance intensity copies
  int* status_host = nullptr;                  // pinned copy of the last call's status word
  cudaStream_t side_stream = nullptr;          // single-CTA probe kernels (CallPtrs::side)
  cudaEvent_t ev_side[4] = {nullptr, nullptr, nullptr, nullptr};
  int inject_alloc_failures = 0;               // adorym_inject_alloc_failures: pending count
  bool timed = false;
  adorym::Serve* serve = nullptr;    // owned; created by the first submit or serve_config
};

namespace adorym {
int get_tables(adorym_ctx* ctx, const adorym_problem& p, Tables* out);   // ctx->mu held
int prepare_kernels(const adorym_problem& p, const char** err);         // attributes, outside capture
const char* status_message(int status);                                 // text of a device status word
void serve_shutdown(adorym_ctx* ctx);
}  // namespace adorym
