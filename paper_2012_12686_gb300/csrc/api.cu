// C ABI entry points: context, object registration, validation, workspace planning, FP64-built
// tables, host-argument staging and the launch sequence of one loss/gradient call.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "engine.h"

namespace adorym {

static const double kPi = 3.14159265358979323846;

static bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }
bool two_pass(int N) { return N >= 256; }

int validate(const adorym_problem& p, const char** err) {
  auto bad = [&](const char* m) {
    *err = m;
    return ADORYM_EINVAL;
  };
  if (p.M < 1 || p.M > 64) return bad("M (probe modes) must be in 1..64");
  if (p.B < 1 || p.B > 65535) return bad("B must be in 1..65535");
  if (p.L < 1) return bad("L must be >= 1");
  if (p.loss != ADORYM_LOSS_LSQ && p.loss != ADORYM_LOSS_POISSON) return bad("loss must be LSQ (0) or Poisson (1)");
  if (!(p.eps >= 0.0)) return bad("eps must be >= 0");
  if (!std::isfinite(p.kdz) || !std::isfinite(p.lambda_dz_over_px2)) return bad("kdz / lambda_dz_over_px2 not finite");
  if (p.checkpoint_every < 0 || p.checkpoint_every > p.L) return bad("checkpoint_every must be in 0..L");
  if (p.gaps)
    for (int j = 0; j + 1 < p.L; ++j)
      if (!std::isfinite(p.gaps[j])) return bad("slice gaps must be finite");
  if (p.farfield) {
    if (!pow2_in(p.N, 8, 1024)) return bad("far field: N must be a power of two in 8..1024");
    if (p.Lz != p.L) return bad("far field: Lz must equal L (the wave crosses every slice)");
    if (p.Ly < 1 || p.Lx < 1) return bad("object dims must be >= 1");
    if (p.tomo && !std::isfinite(p.theta)) return bad("theta not finite");
    if (p.tomo && (p.Lz >= 65536 || p.Lx >= 65536 || (long long)p.Lz * p.Lx >= (1LL << 31) ||
                   (long long)p.Lz * p.Ly * p.Lx >= (1LL << 32)))
      return bad("tomography: Lz and Lx below 65536 and fewer than 2^32 voxels");
  } else {
    if (!pow2_in(p.N, 8, 1024)) return bad("near field: N must be a power of two in 8..1024");
    if (p.tomo) return bad("tomography is defined for the far-field geometry only");
    if (p.Ly != p.N || p.Lx != p.N) return bad("near field: Ly == Lx == N (full-field tiles)");
    if ((long long)p.Lz != (long long)p.B * p.L) return bad("near field: Lz must equal B * L");
    if (p.n_dist < 1 || p.n_dist > 4) return bad("near field: n_dist must be in 1..4");
    for (int d = 0; d < p.n_dist; ++d)
      if (!(p.nf[d] > 0.0) || !std::isfinite(p.nf[d])) return bad("near field: Fresnel numbers must be > 0");
  }
  return ADORYM_OK;
}

std::atomic<unsigned long long> g_kernel_launches{0};

static std::atomic<long long> g_wait_seg{WaitLimits{}.seg}, g_wait_ckpt{WaitLimits{}.ckpt}, g_wait_tma{WaitLimits{}.tma};

WaitLimits wait_limits() {
  WaitLimits w;
  w.seg = g_wait_seg.load(std::memory_order_relaxed);
  w.ckpt = g_wait_ckpt.load(std::memory_order_relaxed);
  w.tma = g_wait_tma.load(std::memory_order_relaxed);
  return w;
}

static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

// SMs of the current device (0 when there is none)
static int device_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

int make_plan(const adorym_problem& p, bool adj, int grads, bool want_loss, Plan* pl, const char** err) {
  int rc = validate(p, err);
  if (rc) return rc;
  Plan q;
  q.p = p;
  q.far = p.farfield != 0;
  q.tomo = p.tomo != 0;
  q.adj = adj;
  q.want_obj = adj && (grads & 1);
  q.want_probe = adj && (grads & 2);
  q.want_offset = adj && (grads & 32) && p.farfield;
  q.want_pos = adj && ((grads & 4) || q.want_offset);
  q.want_nf = adj && (grads & 8) && !p.farfield;
  q.gaps = p.gaps != nullptr && p.L > 1;
  q.want_gaps = adj && (grads & 16) && q.gaps;
  q.want_loss = want_loss;
  q.nd = q.far ? 1 : p.n_dist;
  q.cp = p.checkpoint_every > 0 ? p.checkpoint_every : (int)std::ceil(std::sqrt((double)p.L));
  if (q.cp < 1) q.cp = 1;
  q.ncp = (p.L + q.cp - 1) / q.cp;
  const size_t N = p.N, NN = N * N, B = p.B, M = p.M, f2 = sizeof(float2);
  q.NN = NN;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o += al(bytes);
    return r;
  };
  q.off_phat = take(M * NN * f2);
  if (two_pass(p.N)) {
    q.off_FA = take(B * M * NN * f2);
    if (adj) {
      q.off_FR = take(B * M * NN * f2);
      q.off_ckpt = take(B * M * q.ncp * NN * f2);
      q.off_seg = take(B * M * q.cp * NN * f2);
      q.off_qacc = take(B * M * NN * f2);
      q.off_qsum = take(M * NN * f2);
      q.off_posp = take(B * q.nd * (N / (N == 256 ? 64 : N == 512 ? 32 : 16)) * 3 * sizeof(double));
    }
    q.off_tmp = take(M * NN * f2);
    q.off_far = take(B * (q.far ? 1 : q.nd + 1) * M * NN * f2);
    q.off_gI = take(B * q.nd * NN * sizeof(float));
    q.off_lossp = take(B * q.nd * (NN / 1024) * sizeof(double));
  } else {
    // a batch that fills at most half the SMs gives each position a second CTA that recomputes
    // the next segment while the first reverses the current one (needs two segment slot sets)
    q.pipe = adj && !q.gaps && q.ncp > 1 && q.cp > 1 && 2 * (long long)B <= device_sms();
    if (adj) {
      q.off_ckpt = take(B * M * q.ncp * NN * f2);
      q.off_seg = take(B * M * (q.pipe ? 2 : 1) * q.cp * NN * f2);
      q.off_park = take(B * N * (N + 1) * f2);
      if (!q.far) q.off_fbar = take(B * NN * f2);
      q.off_qacc = take(B * M * NN * f2);
      q.off_qsum = take(M * NN * f2);
    }
    q.off_far = take(B * (q.far ? 1 : q.nd + 1) * M * NN * f2);
    q.off_gI = take(B * q.nd * NN * sizeof(float));
    q.off_lossp = take(B * sizeof(double));
  }
  q.off_loss = take(sizeof(double));
  q.off_box = take(4 * sizeof(int));
  q.off_status = take(sizeof(int));
  if (q.want_offset) {
    q.off_posd = take(B * 2 * sizeof(double));
    q.off_s_goff = take(2 * sizeof(float));
  }
  if (q.want_gaps) {
    const int parts = two_pass(p.N) ? (int)(N / (N == 256 ? 32 : N == 512 ? 16 : 8)) : 1;
    q.off_spck = take(B * M * q.ncp * NN * f2);
    q.off_spseg = take(B * M * q.cp * NN * f2);
    q.off_gapp = take(B * (size_t)(p.L - 1) * parts * sizeof(double));
    q.off_s_ggap = take((size_t)(p.L - 1) * sizeof(float));
  }
  {
    const size_t V = (size_t)p.Lz * p.Ly * p.Lx;
    q.off_T = take(V * f2);
    if (q.want_obj) q.off_grot = take(2 * V * sizeof(double));   // FP64 object-gradient accumulators
    if (q.want_obj && q.tomo) q.off_rtab = take(rot_table_ints(p.Lz, p.Lx) * sizeof(int));
  }
  q.bytes_probe = M * NN * f2;
  q.bytes_pos = B * q.nd * 2 * sizeof(float);
  q.bytes_meas = B * q.nd * NN * sizeof(float);
  q.bytes_iout = q.bytes_meas;
  q.off_s_probe = take(q.bytes_probe);
  q.off_s_pos = take(q.bytes_pos);
  q.off_s_meas = take(q.bytes_meas);
  q.off_s_gprobe = take(q.bytes_probe);
  q.off_s_gpos = take(q.bytes_pos);
  q.off_s_iout = take(q.bytes_iout);
  q.off_s_gnf = take(B * q.nd * sizeof(float));
  q.total = o;
  *pl = q;
  return ADORYM_OK;
}

#ifndef ADORYM_SIDE_STREAM
#define ADORYM_SIDE_STREAM 1
#endif

#ifndef ADORYM_HELPERS
#define ADORYM_HELPERS 1
#endif

size_t helper_ctl_ints(const Plan& q) {
  return q.helpers ? 1 + (size_t)q.p.B * q.p.M * (1 + q.ncp) : 0;
}

void plan_helpers(Plan* pl) {
  Plan& q = *pl;
  const long long B = q.p.B, M = q.p.M, sms = device_sms();
  if (!ADORYM_HELPERS || two_pass(q.p.N) || !q.adj || q.pipe || q.gaps || q.ncp < 2 || q.cp < 2 || B >= sms) return;
  // segments 0..ncp-2 with more than one slice are the tasks; one helper per idle SM, at most one per task
  long long tasks = 0;
  for (int s = 0; s + 1 < q.ncp; ++s) tasks += (std::min((s + 1) * q.cp, q.p.L) - 1 > s * q.cp) ? B * M : 0;
  q.helpers = (int)std::min(sms - B, tasks);
  if (q.helpers <= 0) {
    q.helpers = 0;
    return;
  }
  q.off_hseg = q.total;
  q.total += al((size_t)B * M * (q.ncp - 1) * q.cp * q.NN * sizeof(float2));
  q.off_hctl = q.total;
  q.total += al(helper_ctl_ints(q) * sizeof(int));
}

static std::string table_key(const adorym_problem& p) {
  char buf[256];
  int n = snprintf(buf, sizeof buf, "%d|%.17g|%d", p.N, p.lambda_dz_over_px2, p.farfield ? 0 : p.n_dist);
  if (!p.farfield)
    for (int d = 0; d < p.n_dist; ++d) n += snprintf(buf + n, sizeof buf - n, "|%.17g", p.nf[d]);
  std::string key(buf);
  if (p.gaps && p.L > 1) {
    key += "|gaps";
    for (int j = 0; j + 1 < p.L; ++j) {
      snprintf(buf, sizeof buf, "|%.17g", p.gaps[j]);
      key += buf;
    }
  }
  return key;
}

static double freq(int k, int N) { return (double)(k <= (N - 1) / 2 ? k : k - N) / (double)N; }

static int ngaps(const adorym_problem& p) { return (p.gaps && p.L > 1) ? p.L - 1 : 0; }

size_t table_count(const adorym_problem& p) {
  return (size_t)(3 + (p.farfield ? 0 : p.n_dist)) * p.N + 2 * (size_t)ngaps(p) * p.N;
}

void fill_tables(const adorym_problem& p, float2* h) {
  const int N = p.N, nd = p.farfield ? 0 : p.n_dist;
  for (int m = 0; m < N; ++m) {   // W_N^m = exp(-2 pi i m / N), FP64 argument
    const double a = 2.0 * kPi * (double)m / (double)N;
    h[m] = make_float2((float)std::cos(a), (float)-std::sin(a));
  }
  for (int k = 0; k < N; ++k) {   // paraxial kernel factor exp(i pi c f^2) / N (Eq. paraxial_kernel)
    const double f = freq(k, N), ph = kPi * p.lambda_dz_over_px2 * f * f;
    const float2 v = make_float2((float)(std::cos(ph) / N), (float)(std::sin(ph) / N));
    h[N + k] = v;
    h[2 * N + k] = v;
  }
  for (int d = 0; d < nd; ++d) {  // exp(i pi f^2 / N_F): lambda z / dx^2 = 1 / N_F
    for (int k = 0; k < N; ++k) {
      const double f = freq(k, N), ph = kPi * f * f / p.nf[d];
      h[(size_t)(3 + d) * N + k] = make_float2((float)std::cos(ph), (float)std::sin(ph));
    }
  }
  const int ng = ngaps(p);
  float2* hyj = h + (size_t)(3 + nd) * N;
  for (int j = 0; j < ng; ++j) {   // per-gap factors exp(i pi c_j f^2) / N (variable spacing)
    for (int k = 0; k < N; ++k) {
      const double f = freq(k, N), ph = kPi * p.gaps[j] * f * f;
      const float2 v = make_float2((float)(std::cos(ph) / N), (float)(std::sin(ph) / N));
      hyj[(size_t)j * N + k] = v;
      hyj[(size_t)(ng + j) * N + k] = v;
    }
  }
}

int get_tables(adorym_ctx* ctx, const adorym_problem& p, Tables* out) {
  const std::string key = table_key(p);
  auto it = ctx->tables.find(key);
  if (it != ctx->tables.end()) {
    *out = it->second;
    return ADORYM_OK;
  }
  const int N = p.N, nd = p.farfield ? 0 : p.n_dist;
  std::vector<float2> h(table_count(p));
  fill_tables(p, h.data());
  Tables t;
  t.N = N;
  t.nd = nd;
  t.ngap = ngaps(p);
  cudaError_t e = cudaMalloc(&t.dev, h.size() * sizeof(float2));
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->err = "table allocation failed";
    return ADORYM_ENOMEM;
  }
  e = cudaMemcpy(t.dev, h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    ctx->err = std::string("table upload: ") + cudaGetErrorString(e);
    return ADORYM_EDEVICE;
  }
  ctx->tables[key] = t;
  *out = t;
  return ADORYM_OK;
}

int enqueue(const Plan& pl, const Object& obj, const Tables& tab, const CallPtrs& c, char* ws, cudaStream_t s,
            std::string* err, cudaEvent_t ev_start, cudaEvent_t ev_stop) {
  const adorym_problem& p = pl.p;
  auto W = [&](size_t off) { return ws + off; };
  auto chk = [&](cudaError_t e, const char* what) {
    if (e == cudaSuccess) return ADORYM_OK;
    *err = std::string(what) + ": " + cudaGetErrorString(e);
    return ADORYM_EDEVICE;
  };
  double *gd = nullptr, *gb = nullptr;
  const size_t V = (size_t)p.Lz * p.Ly * p.Lx;
  const double cth = std::cos(p.theta), sth = std::sin(p.theta);
  int rc;
  float2* T = reinterpret_cast<float2*>(W(pl.off_T));
  int* box = reinterpret_cast<int*>(W(pl.off_box));
  int* status = c.status ? c.status : reinterpret_cast<int*>(W(pl.off_status));
  bool join_side = false;   // the call's stream waits for the side stream's last kernels
  if (!c.status && (rc = chk(cudaMemsetAsync(status, 0, sizeof(int), s), "status"))) return rc;
  float2* phat = reinterpret_cast<float2*>(W(pl.off_phat));
  // the probe transform needs only the probe: on the side stream it overlaps the passes below
  const bool side = c.side && !two_pass(p.N);
  if (side && pl.far) {
    if ((rc = chk(cudaEventRecord(c.ev_side[0], s), "fork"))) return rc;
    if ((rc = chk(cudaStreamWaitEvent(c.side, c.ev_side[0], 0), "fork"))) return rc;
    if ((rc = chk(launch_probe_hat(p.N, p.M, c.probe, phat, tab.tw(), c.side), "probe_hat"))) return rc;
    if ((rc = chk(cudaEventRecord(c.ev_side[1], c.side), "join"))) return rc;
  }
  int* hctl = pl.helpers ? reinterpret_cast<int*>(W(pl.off_hctl)) : nullptr;
  if ((rc = chk(launch_bbox(c.pos, p.B, p.N, p.Ly, p.Lx, pl.far ? 1 : 0, pl.tomo ? 1 : 0, box, 2 * p.B * pl.nd, status,
                            s, hctl, (int)helper_ctl_ints(pl)),
                "bbox")))
    return rc;
  // near field with one probe mode: one term per voxel and call, added in place by the kernels
  const bool direct = pl.want_obj && !pl.far && p.M == 1;
  if (pl.want_obj && !direct) {
    // the scatter-add over overlapping positions is a reduction: accumulate it in FP64 (the
    // accumulators are zeroed over the box by the transmission pass)
    double* acc = reinterpret_cast<double*>(W(pl.off_grot));
    gd = acc;
    gb = acc + V;
  }
  if ((rc = chk(launch_transmission(obj.d, obj.b, T, p.Lz, p.Ly, p.Lx, (float)p.kdz, pl.tomo ? 1 : 0, (float)cth,
                                    (float)sth, box, gd, gb, s),
                "transmission")))
    return rc;
  // the fused kernel reads the measured intensities: wait for their copy before it (the pre-kernels
  // above and the probe transform do not read them); the two-pass sequence waits inside, before
  // its detector passes
  auto wait_meas = [&]() -> int {
    return c.meas_ready ? chk(cudaStreamWaitEvent(s, c.meas_ready, 0), "wait for intensities") : ADORYM_OK;
  };
  if (two_pass(p.N)) {
    TPArgs t{};
    t.N = p.N;
    t.L = p.L;
    t.M = p.M;
    t.B = p.B;
    t.Ly = p.Ly;
    t.Lx = p.Lx;
    t.cp = pl.cp;
    t.ncp = pl.ncp;
    t.nd = pl.nd;
    t.loss = p.loss;
    t.farfield = pl.far ? 1 : 0;
    t.adj = pl.adj ? 1 : 0;
    t.eps = (float)p.eps;
    t.kdz = (float)p.kdz;
    t.wait_tma = wait_limits().tma;
    t.inv_npix = 1.0 / ((double)p.B * pl.nd * (double)pl.NN);
    t.T = T;
    t.probe = c.probe;
    t.phat = phat;
    t.phat_w = phat;
    t.pos = c.pos;
    t.I_meas = c.I_meas;
    t.I_out = c.I_out;
    t.tw = tab.tw();
    t.hy = tab.hy();
    t.hx = tab.hx();
    t.hd = pl.far ? nullptr : tab.hd();
    t.hyj = tab.hyj();
    t.hxj = tab.hxj();
    t.FA = reinterpret_cast<float2*>(W(pl.off_FA));
    t.far = reinterpret_cast<float2*>(W(pl.off_far));
    t.gI = reinterpret_cast<float*>(W(pl.off_gI));
    t.lossp = reinterpret_cast<double*>(W(pl.off_lossp));
    t.status = status;
    t.tmp = reinterpret_cast<float2*>(W(pl.off_tmp));
    if (pl.adj) {
      t.FR = reinterpret_cast<float2*>(W(pl.off_FR));
      t.ckpt = reinterpret_cast<float2*>(W(pl.off_ckpt));
      t.seg = reinterpret_cast<float2*>(W(pl.off_seg));
      t.qacc = pl.want_probe ? reinterpret_cast<float2*>(W(pl.off_qacc)) : nullptr;
      t.qsum = reinterpret_cast<float2*>(W(pl.off_qsum));
      t.posp = (pl.want_pos || pl.want_nf) ? reinterpret_cast<double*>(W(pl.off_posp)) : nullptr;
      t.gnf = pl.want_nf ? c.g_nf : nullptr;
      for (int d = 0; d < 4; ++d) t.nf[d] = p.nf[d];
      if (pl.want_gaps) {
        t.spec_out = reinterpret_cast<float2*>(W(pl.off_spck));    // spectra: [B][M][ncp] then [B][M][cp]
        t.spec_in = reinterpret_cast<float2*>(W(pl.off_spseg));
        t.gapp = reinterpret_cast<double*>(W(pl.off_gapp));
        t.ggap = c.g_gaps;
      }
      t.gd = pl.want_obj ? gd : nullptr;
      t.gb = pl.want_obj ? gb : nullptr;
      t.gdf = direct ? c.gd : nullptr;
      t.gbf = direct ? c.gb : nullptr;
      t.gpos = pl.want_pos ? c.g_pos : nullptr;
      t.gposd = pl.want_offset ? reinterpret_cast<double*>(W(pl.off_posd)) : nullptr;
      t.g_probe = pl.want_probe ? c.g_probe : nullptr;
      t.loss_out = c.loss;
    }
    if ((rc = chk(launch_twopass(t, s, ev_start, ev_stop, c.meas_ready, c.meas_part, c.n_meas_part), "two-pass")))
      return rc;
  } else {
    if (pl.far) {
      rc = side ? chk(cudaStreamWaitEvent(s, c.ev_side[1], 0), "join")
                : chk(launch_probe_hat(p.N, p.M, c.probe, phat, tab.tw(), s), "probe_hat");
      if (rc) return rc;
    }
    PathArgs a{};
    a.N = p.N;
    a.L = p.L;
    a.M = p.M;
    a.B = p.B;
    a.Ly = p.Ly;
    a.Lx = p.Lx;
    a.cp = pl.cp;
    a.ncp = pl.ncp;
    a.loss = p.loss;
    a.adj = pl.adj ? 1 : 0;
    a.n_dist = pl.nd;
    a.pipe = pl.pipe ? 1 : 0;
    a.eps = (float)p.eps;
    a.kdz = (float)p.kdz;
    a.wait_seg = wait_limits().seg;
    a.wait_ckpt = wait_limits().ckpt;
    a.inv_npix = 1.0 / ((double)p.B * pl.nd * (double)pl.NN);
    a.T = T;
    a.probe = c.probe;
    a.phat = phat;
    a.pos = c.pos;
    a.I_meas = c.I_meas;
    a.I_out = c.I_out;
    a.tw = tab.tw();
    a.hy = tab.hy();
    a.hx = tab.hx();
    a.hd = pl.far ? nullptr : tab.hd();
    a.hyj = tab.hyj();
    a.hxj = tab.hxj();
    if (pl.adj) {
      a.ckpt = reinterpret_cast<float2*>(W(pl.off_ckpt));
      a.seg = reinterpret_cast<float2*>(W(pl.off_seg));
      a.park = reinterpret_cast<float2*>(W(pl.off_park));
      a.fbar = pl.far ? nullptr : reinterpret_cast<float2*>(W(pl.off_fbar));
      a.qacc = pl.want_probe ? reinterpret_cast<float2*>(W(pl.off_qacc)) : nullptr;
      a.gd = pl.want_obj ? gd : nullptr;
      a.gb = pl.want_obj ? gb : nullptr;
      a.gdf = direct ? c.gd : nullptr;
      a.gbf = direct ? c.gb : nullptr;
      a.gpos = pl.want_pos ? c.g_pos : nullptr;
      a.gposd = pl.want_offset ? reinterpret_cast<double*>(W(pl.off_posd)) : nullptr;
      a.gnf = pl.want_nf ? c.g_nf : nullptr;
      for (int d = 0; d < 4; ++d) a.nf[d] = p.nf[d];
      if (pl.want_gaps) {
        a.spck = reinterpret_cast<float2*>(W(pl.off_spck));
        a.spseg = reinterpret_cast<float2*>(W(pl.off_spseg));
        a.gapp = reinterpret_cast<double*>(W(pl.off_gapp));
      }
    }
    if (pl.helpers) {
      a.helpers = pl.helpers;
      a.hseg = reinterpret_cast<float2*>(W(pl.off_hseg));
      a.hnext = hctl;
      a.hprog = hctl + 1;
      a.hflag = hctl + 1 + (size_t)p.B * p.M;
    }
    a.far = reinterpret_cast<float2*>(W(pl.off_far));
    a.gI = reinterpret_cast<float*>(W(pl.off_gI));
    a.lossp = reinterpret_cast<double*>(W(pl.off_lossp));
    if ((rc = wait_meas())) return rc;
    if (ev_start) cudaEventRecord(ev_start, s);
    if ((rc = chk(launch_path(a, pl.far ? 1 : 0, s), "path"))) return rc;
    if (ev_stop) cudaEventRecord(ev_stop, s);
    if (pl.want_gaps && c.g_gaps) {
      if ((rc = chk(launch_gap_final(a.gapp, p.B, p.L - 1, 1, c.g_gaps, s), "gap_final"))) return rc;
    }
    if (pl.adj && (pl.want_probe || c.loss)) {
      // the probe-gradient kernels (one CTA per mode) run beside the object-gradient pass
      cudaStream_t sp = side ? c.side : s;
      if (side) {
        if ((rc = chk(cudaEventRecord(c.ev_side[2], s), "fork"))) return rc;
        if ((rc = chk(cudaStreamWaitEvent(c.side, c.ev_side[2], 0), "fork"))) return rc;
      }
      if ((rc = chk(launch_probe_grad(p.N, p.M, p.B, pl.far ? 1 : 0, a.qacc, reinterpret_cast<float2*>(W(pl.off_qsum)),
                                      pl.want_probe ? c.g_probe : nullptr, tab.tw(), a.lossp, a.inv_npix, c.loss, sp),
                    "probe_grad")))
        return rc;
      if (side) {
        if ((rc = chk(cudaEventRecord(c.ev_side[3], c.side), "join"))) return rc;
        join_side = true;
      }
    }
  }
  if (pl.want_offset && c.g_offset) {
    if ((rc = chk(launch_offset_sum(reinterpret_cast<double*>(W(pl.off_posd)), p.B, c.g_offset, s), "offset_sum")))
      return rc;
  }
  if (pl.want_obj && !direct) {
    if (pl.tomo)
      rc = chk(launch_rotate_adj(gd, gb, c.gd, c.gb, p.Lz, p.Ly, p.Lx, (float)cth, (float)sth, box,
                                 reinterpret_cast<int*>(W(pl.off_rtab)), s),
               "rotate_adj");
    else
      rc = chk(launch_grad_add(gd, gb, c.gd, c.gb, p.Lz, p.Ly, p.Lx, box, s), "grad_add");
    if (rc) return rc;
  }
  if (join_side && (rc = chk(cudaStreamWaitEvent(s, c.ev_side[3], 0), "join"))) return rc;
  return ADORYM_OK;
}

int prepare_kernels(const adorym_problem& p, const char** err) {
  cudaError_t e = two_pass(p.N) ? prepare_twopass(p.N) : prepare_path(p.N, p.farfield ? 1 : 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *err = "kernel attributes could not be set";
    return ADORYM_EDEVICE;
  }
  return ADORYM_OK;
}

const char* status_message(int status) {
  return (status & STATUS_BAD_POSITION)   ? "a position or hologram shift is not finite or lies beyond +-2^24 px"
         : (status & STATUS_WAIT_TIMEOUT) ? "a device-side wait for a tile copy timed out"
                                          : "invalid input data";
}

}  // namespace adorym

using namespace adorym;

static int fail(adorym_ctx* ctx, int rc, const std::string& m) {
  ctx->err = m;
  return rc;
}

static int cuda_fail(adorym_ctx* ctx, cudaError_t e, const char* what) {
  cudaGetLastError();
  ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
  return ADORYM_EDEVICE;
}

// 1 = device (or managed), 0 = host (pinned or pageable), -1 = null
static int ptr_kind(const void* p) {
  if (!p) return -1;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) ? 1 : 0;
}

static int ensure_ws(adorym_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_cap) return ADORYM_OK;
  if (ctx->inject_alloc_failures > 0) {   // injected: fail before the current workspace is touched
    --ctx->inject_alloc_failures;
    return fail(ctx, ADORYM_ENOMEM, "injected workspace allocation failure");
  }
  cudaStreamSynchronize(ctx->stream);
  if (ctx->ws) cudaFree(ctx->ws);
  ctx->ws = nullptr;
  ctx->ws_cap = 0;
  const size_t cap = bytes + bytes / 8;
  cudaError_t e = cudaMalloc(&ctx->ws, cap);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, ADORYM_ENOMEM, "workspace allocation of " + std::to_string(cap) + " bytes failed");
  }
  ctx->ws_cap = cap;
  return ADORYM_OK;
}

extern "C" {

int adorym_create(adorym_ctx** out, int device, void* stream) {
  if (!out) return ADORYM_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return ADORYM_EDEVICE;
  }
  if (cudaSetDevice(device) != cudaSuccess) return ADORYM_EDEVICE;
  adorym_ctx* c = new adorym_ctx();
  c->device = device;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  *out = c;
  return ADORYM_OK;
}

void adorym_destroy(adorym_ctx* ctx) {
  if (!ctx) return;
  serve_shutdown(ctx);
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->ws) cudaFree(ctx->ws);
  for (auto& kv : ctx->tables) cudaFree(kv.second.dev);
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  if (ctx->copy_stream) {
    cudaStreamSynchronize(ctx->copy_stream);
    cudaStreamDestroy(ctx->copy_stream);
  }
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->status_host) cudaFreeHost(ctx->status_host);
  if (ctx->ev_meas) cudaEventDestroy(ctx->ev_meas);
  for (cudaEvent_t e : ctx->ev_meas_d)
    if (e) cudaEventDestroy(e);
  if (ctx->side_stream) {
    cudaStreamSynchronize(ctx->side_stream);
    cudaStreamDestroy(ctx->side_stream);
  }
  for (cudaEvent_t e : ctx->ev_side)
    if (e) cudaEventDestroy(e);
  delete ctx;
}

const char* adorym_last_error(adorym_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int adorym_inject_alloc_failures(adorym_ctx* ctx, int count) {
  if (!ctx || count < 0) return ADORYM_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->inject_alloc_failures = count;
  return ADORYM_OK;
}

uint64_t adorym_kernel_launches(void) { return g_kernel_launches.load(std::memory_order_relaxed); }

int adorym_set_wait_limits(int64_t segment_cycles, int64_t checkpoint_cycles, int64_t tile_copy_cycles) {
  if (segment_cycles < ADORYM_WAIT_DEFAULT || checkpoint_cycles < ADORYM_WAIT_DEFAULT ||
      tile_copy_cycles < ADORYM_WAIT_GIVE_UP)
    return ADORYM_EINVAL;
  const WaitLimits d;
  g_wait_seg.store(segment_cycles == ADORYM_WAIT_DEFAULT ? d.seg : segment_cycles);
  g_wait_ckpt.store(checkpoint_cycles == ADORYM_WAIT_DEFAULT ? d.ckpt : checkpoint_cycles);
  g_wait_tma.store(tile_copy_cycles == ADORYM_WAIT_DEFAULT ? d.tma : tile_copy_cycles == ADORYM_WAIT_GIVE_UP ? -1
                                                                                                         : tile_copy_cycles);
  return ADORYM_OK;
}

int adorym_check(adorym_ctx* ctx) {
  if (!ctx) return ADORYM_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!ctx->status_host) return ADORYM_OK;   // no call yet
  cudaSetDevice(ctx->device);
  const cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
  if (*ctx->status_host) return fail(ctx, ADORYM_EDATA, status_message(*ctx->status_host));
  return ADORYM_OK;
}

int adorym_register_object(adorym_ctx* ctx, const float* delta, const float* beta, int Lz, int Ly, int Lx,
                           int* obj_id) {
  if (!ctx || !obj_id) return ADORYM_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (Lz < 1 || Ly < 1 || Lx < 1) return fail(ctx, ADORYM_EINVAL, "object dims must be >= 1");
  if (ptr_kind(delta) != 1 || ptr_kind(beta) != 1)
    return fail(ctx, ADORYM_EINVAL, "object volumes must be device memory");
  Object o;
  o.d = delta;
  o.b = beta;
  o.Lz = Lz;
  o.Ly = Ly;
  o.Lx = Lx;
  const int id = ctx->next_obj++;
  ctx->objects[id] = o;
  *obj_id = id;
  return ADORYM_OK;
}

int adorym_unregister_object(adorym_ctx* ctx, int obj_id) {
  if (!ctx) return ADORYM_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!ctx->objects.erase(obj_id)) return fail(ctx, ADORYM_ENOENT, "unknown object id");
  return ADORYM_OK;
}

int adorym_workspace_bytes(const adorym_problem* p, int grads, uint64_t* bytes) {
  if (!p || !bytes) return ADORYM_EINVAL;
  Plan pl;
  const char* err = "";
  int rc = make_plan(*p, true, grads, true, &pl, &err);
  if (rc) return rc;
  *bytes = pl.total;
  return ADORYM_OK;
}

static int run_call(adorym_ctx* ctx, const adorym_problem* p, int obj_id, const float* probe, const float* pos,
                    const float* I_meas, double* loss_out, float* g_delta, float* g_beta, float* g_probe,
                    float* g_pos, float* I_out, bool adj, float* g_nf = nullptr, float* g_gaps = nullptr,
                    float* g_offset = nullptr) {
  if (!ctx) return ADORYM_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!p) return fail(ctx, ADORYM_EINVAL, "null problem");
  if (!probe || !pos) return fail(ctx, ADORYM_EINVAL, "probe and pos are required");
  if (adj && !I_meas) return fail(ctx, ADORYM_EINVAL, "I_meas is required for loss_grad");
  if (!adj && !I_out) return fail(ctx, ADORYM_EINVAL, "I_out is required for forward");
  if ((g_delta == nullptr) != (g_beta == nullptr))
    return fail(ctx, ADORYM_EINVAL, "g_delta and g_beta must both be given or both be NULL");
  auto it = ctx->objects.find(obj_id);
  if (it == ctx->objects.end()) return fail(ctx, ADORYM_ENOENT, "unknown object id");
  const Object& obj = it->second;
  if (obj.Lz != p->Lz || obj.Ly != p->Ly || obj.Lx != p->Lx)
    return fail(ctx, ADORYM_EINVAL, "problem Lz/Ly/Lx differ from the registered object");
  if (g_delta && (ptr_kind(g_delta) != 1 || ptr_kind(g_beta) != 1))
    return fail(ctx, ADORYM_EINVAL, "g_delta / g_beta must be device memory");
  const int grads = (g_delta ? 1 : 0) | (g_probe ? 2 : 0) | (g_pos ? 4 : 0) | (g_nf ? 8 : 0) | (g_gaps ? 16 : 0) |
                    (g_offset ? 32 : 0);
  if (g_offset && !p->farfield)
    return fail(ctx, ADORYM_EINVAL, "g_offset (per-angle position offset) is defined for the far-field geometry only");
  if (g_gaps && !(p->gaps && p->L > 1))
    return fail(ctx, ADORYM_EINVAL, "g_gaps needs variable slice spacing (gaps) and L > 1");
  if (g_nf && p->farfield) return fail(ctx, ADORYM_EINVAL, "g_nf is defined for the near-field geometry only");
  Plan pl;
  const char* msg = "";
  int rc = make_plan(*p, adj, grads, loss_out != nullptr, &pl, &msg);
  if (rc) return fail(ctx, rc, msg);
  std::string err;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "set device");
  plan_helpers(&pl);
  Tables tab;
  if ((rc = get_tables(ctx, *p, &tab))) return rc;
  if ((rc = prepare_kernels(*p, &msg))) return fail(ctx, rc, msg);
  if ((rc = ensure_ws(ctx, pl.total))) return rc;
  char* ws = ctx->ws;
  cudaStream_t s = ctx->stream;
  bool sync_after = false;
  CallPtrs c;
  auto stage_in = [&](const void* src, size_t off, size_t bytes) -> const void* {
    if (ptr_kind(src) == 1) return src;
    cudaMemcpyAsync(ws + off, src, bytes, cudaMemcpyHostToDevice, s);
    return ws + off;
  };
  c.probe = reinterpret_cast<const float2*>(stage_in(probe, pl.off_s_probe, pl.bytes_probe));
  c.pos = reinterpret_cast<const float*>(stage_in(pos, pl.off_s_pos, pl.bytes_pos));
  if (I_meas && ptr_kind(I_meas) != 1) {
    // host intensities: copied on a side stream that starts once the stream's earlier work (which
    // may still read the staging area) is done, overlapping this call's pre-kernels
    if (!ctx->copy_stream) {
      if (cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&ctx->ev_meas, cudaEventDisableTiming) != cudaSuccess)
        return cuda_fail(ctx, cudaGetLastError(), "copy stream");
    }
    cudaEventRecord(ctx->ev_fork, s);
    cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_fork, 0);
    c.I_meas = reinterpret_cast<const float*>(ws + pl.off_s_meas);
    c.meas_ready = ctx->ev_meas;
    if (two_pass(p->N) && !pl.far && pl.nd > 1) {
      // one strided copy per distance ([B] rows of N^2 values at a pitch of n_dist N^2), each
      // with its own event: the detector pass of distance d starts once its rows have arrived
      if (!ctx->ev_meas_d[0]) {
        bool ok = true;
        for (cudaEvent_t& e : ctx->ev_meas_d) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
        if (!ok) return cuda_fail(ctx, cudaGetLastError(), "copy events");
      }
      const size_t row = pl.NN * sizeof(float), pitch = (size_t)pl.nd * row;
      for (int d = 0; d < pl.nd; ++d) {
        cudaMemcpy2DAsync(ws + pl.off_s_meas + d * row, pitch, reinterpret_cast<const char*>(I_meas) + d * row, pitch, row,
                          (size_t)p->B, cudaMemcpyHostToDevice, ctx->copy_stream);
        cudaEventRecord(ctx->ev_meas_d[d], ctx->copy_stream);
      }
      c.meas_ready = ctx->ev_meas_d[pl.nd - 1];   // the copy stream is in order: the last part
      c.meas_part = ctx->ev_meas_d;
      c.n_meas_part = pl.nd;
    } else {
      cudaMemcpyAsync(ws + pl.off_s_meas, I_meas, pl.bytes_meas, cudaMemcpyHostToDevice, ctx->copy_stream);
      cudaEventRecord(ctx->ev_meas, ctx->copy_stream);
    }
  } else if (I_meas) {
    c.I_meas = I_meas;
  }
  c.gd = g_delta;
  c.gb = g_beta;
  const bool host_loss = loss_out && ptr_kind(loss_out) == 0;
  const bool host_gprobe = g_probe && ptr_kind(g_probe) == 0;
  const bool host_gpos = g_pos && ptr_kind(g_pos) == 0;
  const bool host_iout = I_out && ptr_kind(I_out) == 0;
  const bool host_gnf = g_nf && ptr_kind(g_nf) == 0;
  const bool host_ggap = g_gaps && ptr_kind(g_gaps) == 0;
  const bool host_goff = g_offset && ptr_kind(g_offset) == 0;
  if (g_offset) c.g_offset = host_goff ? reinterpret_cast<float*>(ws + pl.off_s_goff) : g_offset;
  if (g_gaps) c.g_gaps = host_ggap ? reinterpret_cast<float*>(ws + pl.off_s_ggap) : g_gaps;
  if (g_nf) c.g_nf = host_gnf ? reinterpret_cast<float*>(ws + pl.off_s_gnf) : g_nf;
  c.loss = loss_out ? (host_loss ? reinterpret_cast<double*>(ws + pl.off_loss) : loss_out) : nullptr;
  if (g_probe) {
    if (host_gprobe) {
      cudaMemcpyAsync(ws + pl.off_s_gprobe, g_probe, pl.bytes_probe, cudaMemcpyHostToDevice, s);
      c.g_probe = reinterpret_cast<float2*>(ws + pl.off_s_gprobe);
    } else {
      c.g_probe = reinterpret_cast<float2*>(g_probe);
    }
  }
  if (g_pos) c.g_pos = host_gpos ? reinterpret_cast<float*>(ws + pl.off_s_gpos) : g_pos;
  if (I_out) c.I_out = host_iout ? reinterpret_cast<float*>(ws + pl.off_s_iout) : I_out;
  if (ctx->timing && !ctx->ev0) {
    cudaEventCreate(&ctx->ev0);
    cudaEventCreate(&ctx->ev1);
  }
  if (ADORYM_SIDE_STREAM && !two_pass(p->N)) {
    if (!ctx->side_stream) {
      // highest priority: the one-CTA probe kernels on it must not queue behind the many-block
      // box kernels of the call's stream that they overlap (transmission before the fused kernel,
      // object-gradient add after it)
      int least = 0, greatest = 0;
      bool ok = cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess;
      ok = ok && cudaStreamCreateWithPriority(&ctx->side_stream, cudaStreamNonBlocking, greatest) == cudaSuccess;
      for (cudaEvent_t& e : ctx->ev_side) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
      if (!ok) return cuda_fail(ctx, cudaGetLastError(), "side stream");
    }
    c.side = ctx->side_stream;
    for (int i = 0; i < 4; ++i) c.ev_side[i] = ctx->ev_side[i];
  }
  if ((rc = enqueue(pl, obj, tab, c, ws, s, &err, ctx->timing ? ctx->ev0 : nullptr, ctx->timing ? ctx->ev1 : nullptr)))
    return fail(ctx, rc, err);
  ctx->timed = ctx->timing;
  if (host_loss) {
    cudaMemcpyAsync(loss_out, c.loss, sizeof(double), cudaMemcpyDeviceToHost, s);
    sync_after = true;
  }
  if (host_gprobe) {
    cudaMemcpyAsync(g_probe, c.g_probe, pl.bytes_probe, cudaMemcpyDeviceToHost, s);
    sync_after = true;
  }
  if (host_gpos) {
    cudaMemcpyAsync(g_pos, c.g_pos, pl.bytes_pos, cudaMemcpyDeviceToHost, s);
    sync_after = true;
  }
  if (host_iout) {
    cudaMemcpyAsync(I_out, c.I_out, pl.bytes_iout, cudaMemcpyDeviceToHost, s);
    sync_after = true;
  }
  if (host_gnf) {
    cudaMemcpyAsync(g_nf, c.g_nf, (size_t)p->B * pl.nd * sizeof(float), cudaMemcpyDeviceToHost, s);
    sync_after = true;
  }
  if (host_ggap) {
    cudaMemcpyAsync(g_gaps, c.g_gaps, (size_t)(p->L - 1) * sizeof(float), cudaMemcpyDeviceToHost, s);
    sync_after = true;
  }
  if (host_goff) {
    cudaMemcpyAsync(g_offset, c.g_offset, 2 * sizeof(float), cudaMemcpyDeviceToHost, s);
    sync_after = true;
  }
  // the call's status word goes to a pinned host int (read by adorym_check, or below)
  if (!ctx->status_host) {
    void* h = nullptr;
    if (cudaHostAlloc(&h, sizeof(int), cudaHostAllocDefault) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "status");
    ctx->status_host = static_cast<int*>(h);
  }
  cudaMemcpyAsync(ctx->status_host, ws + pl.off_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "enqueue");
  if (sync_after) {
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
    if (*ctx->status_host) return fail(ctx, ADORYM_EDATA, status_message(*ctx->status_host));
  }
  return ADORYM_OK;
}

int adorym_enable_kernel_timing(adorym_ctx* ctx, int enable) {
  if (!ctx) return ADORYM_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->timing = enable != 0;
  return ADORYM_OK;
}

int adorym_kernel_ms(adorym_ctx* ctx, float* path_ms) {
  if (!ctx || !path_ms) return ADORYM_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!ctx->timed || !ctx->ev1) return fail(ctx, ADORYM_ENOENT, "no timed call yet");
  cudaError_t e = cudaEventSynchronize(ctx->ev1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(path_ms, ctx->ev0, ctx->ev1);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel timing");
  return ADORYM_OK;
}

int adorym_forward(adorym_ctx* ctx, const adorym_problem* p, int obj_id, const float* probe, const float* pos,
                   float* I_out) {
  return run_call(ctx, p, obj_id, probe, pos, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, I_out, false);
}

int adorym_loss_grad(adorym_ctx* ctx, const adorym_problem* p, int obj_id, const float* probe, const float* pos,
                     const float* I_meas, double* loss_out, float* g_delta, float* g_beta, float* g_probe,
                     float* g_pos, float* I_out) {
  return run_call(ctx, p, obj_id, probe, pos, I_meas, loss_out, g_delta, g_beta, g_probe, g_pos, I_out, true);
}

int adorym_regularize(adorym_ctx* ctx, int obj_id, const adorym_reg* r, double* loss_out, float* g_delta,
                      float* g_beta) {
  if (!ctx) return ADORYM_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!r) return fail(ctx, ADORYM_EINVAL, "null regularizer description");
  if ((g_delta == nullptr) != (g_beta == nullptr))
    return fail(ctx, ADORYM_EINVAL, "g_delta and g_beta must both be given or both be NULL");
  auto it = ctx->objects.find(obj_id);
  if (it == ctx->objects.end()) return fail(ctx, ADORYM_ENOENT, "unknown object id");
  const Object& o = it->second;
  const void* dev_ptrs[] = {g_delta, g_beta, r->w_delta, r->w_beta};
  for (const void* q : dev_ptrs)
    if (q && ptr_kind(q) != 1) return fail(ctx, ADORYM_EINVAL, "gradient and weight arrays must be device memory");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "set device");
  const size_t n = (size_t)o.Lz * o.Ly * o.Lx;
  const size_t need = al(reg_parts(n) * sizeof(double)) + al(sizeof(double));
  int rc = ensure_ws(ctx, need);
  if (rc) return rc;
  double* part = reinterpret_cast<double*>(ctx->ws);
  double* dloss = reinterpret_cast<double*>(ctx->ws + al(reg_parts(n) * sizeof(double)));
  const bool host_loss = loss_out && ptr_kind(loss_out) == 0;
  double* lp = loss_out ? (host_loss ? dloss : loss_out) : nullptr;
  cudaError_t e = launch_regularize(o.d, o.b, r->w_delta, r->w_beta, o.Lz, o.Ly, o.Lx, r->alpha_delta, r->alpha_beta,
                                    r->gamma_tv, g_delta, g_beta, part, lp, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "regularize");
  if (host_loss) {
    cudaMemcpyAsync(loss_out, dloss, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
  }
  return ADORYM_OK;
}

int adorym_l1_weights(adorym_ctx* ctx, int obj_id, double eps, float* w_delta, float* w_beta) {
  if (!ctx) return ADORYM_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->objects.find(obj_id);
  if (it == ctx->objects.end()) return fail(ctx, ADORYM_ENOENT, "unknown object id");
  if (!(eps > 0.0)) return fail(ctx, ADORYM_EINVAL, "eps must be > 0");
  if (ptr_kind(w_delta) != 1 || ptr_kind(w_beta) != 1) return fail(ctx, ADORYM_EINVAL, "weights must be device memory");
  const Object& o = it->second;
  const size_t n = (size_t)o.Lz * o.Ly * o.Lx;
  int rc = ensure_ws(ctx, al(reg_parts(n) * sizeof(float)));
  if (rc) return rc;
  float* part = reinterpret_cast<float*>(ctx->ws);
  cudaError_t e = launch_l1_weights(o.d, n, (float)eps, part, w_delta, ctx->stream);
  if (e == cudaSuccess) e = launch_l1_weights(o.b, n, (float)eps, part, w_beta, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "l1 weights");
  return ADORYM_OK;
}

int adorym_loss_grad_ext(adorym_ctx* ctx, const adorym_problem* p, int obj_id, const float* probe, const float* pos,
                         const float* I_meas, const adorym_grads* out) {
  if (!out) return run_call(ctx, p, obj_id, probe, pos, I_meas, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                            true);
  return run_call(ctx, p, obj_id, probe, pos, I_meas, out->loss, out->g_delta, out->g_beta, out->g_probe, out->g_pos,
                  out->I_out, true, out->g_nf, out->g_gaps, out->g_offset);
}

}  // extern "C"
