// adorym_loss_grad_noalloc: the loss/gradient call for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: plug-ins of host frameworks that own every device
// allocation through their own pool, or real-time loops where an allocation (and the device
// synchronisation it can bring) is not acceptable.  This entry point therefore draws all of its
// workspace -- checkpoints, segment buffers, far-field and loss partials, probe-gradient partials
// and the twiddle/propagator tables -- from one file-scope device array of fixed size, and calls
// no cudaMalloc, cudaFree or other allocating routine.  The caller still passes every input and
// output, as device pointers.  The tables are computed on the device by a small kernel on the
// caller's stream (FP64 arguments, rounded once to FP32), so the call reads no host memory after
// it returns.
//
// The array (ADORYM_NOALLOC_SCRATCH_BYTES) is reserved on every GPU that loads this code and
// stays reserved until the process exits.  Its device address is looked up once per device with
// cudaGetSymbolAddress (the name is only a host-side stand-in for the device address), on the
// first call made with that device current.  All calls share the array and it keeps the last
// call's contents: the parts that must start at zero are cleared on the stream by each call, and
// calls whose work overlaps on the GPU (different streams, or several host threads) race on it
// and must be serialised by the caller.
#include <mutex>

#include "engine.h"

namespace {

constexpr size_t kScratchBytes = ADORYM_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
char* g_scratch_ptr[kMaxDevices] = {};

// device address of g_scratch for the current device (looked up once per device)
int scratch_address(int dev, char** out) {
  if (dev < 0 || dev >= kMaxDevices) return ADORYM_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return ADORYM_EDEVICE;
    }
    g_scratch_ptr[dev] = static_cast<char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return ADORYM_OK;
}

bool on_device(const void* p) {
  if (!p) return true;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// The FP64-built tables of a uniform-spacing problem (the layout of adorym::Tables): W_N^m =
// exp(-2 pi i m / N), the paraxial factors exp(i pi c f^2) / N twice (y, x), and per detector
// distance exp(i pi f^2 / N_F), f = fftfreq(N) in cycles per pixel.
__global__ void k_noalloc_tables(float2* out, int N, double c, int nd, double nf0, double nf1, double nf2,
                                 double nf3) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (3 + nd) * N) return;
  const int row = i / N, k = i - row * N;
  const double f = (double)(k <= (N - 1) / 2 ? k : k - N) / (double)N;
  double sn, cs;
  if (row == 0) {
    sincospi(2.0 * (double)k / (double)N, &sn, &cs);
    out[i] = make_float2((float)cs, (float)-sn);
  } else if (row <= 2) {
    sincospi(c * f * f, &sn, &cs);
    out[i] = make_float2((float)(cs / N), (float)(sn / N));
  } else {
    const int d = row - 3;
    const double nf = d == 0 ? nf0 : d == 1 ? nf1 : d == 2 ? nf2 : nf3;
    sincospi(f * f / nf, &sn, &cs);
    out[i] = make_float2((float)cs, (float)sn);
  }
}

}  // namespace

using namespace adorym;

extern "C" int adorym_loss_grad_noalloc(void* cuda_stream, const adorym_problem* p, const float* delta,
                                        const float* beta, const float* probe, const float* pos,
                                        const float* I_meas, double* loss_out, float* g_delta, float* g_beta,
                                        float* g_probe, float* g_pos, float* I_out, int* status) {
  if (!p || !delta || !beta || !probe || !pos || !I_meas) return ADORYM_EINVAL;
  if (p->gaps && p->L > 1) return ADORYM_EINVAL;   // variable slice spacing: not offered by this entry point
  if ((g_delta == nullptr) != (g_beta == nullptr)) return ADORYM_EINVAL;
  const void* ptrs[] = {delta, beta, probe, pos, I_meas, loss_out, g_delta, g_beta, g_probe, g_pos, I_out, status};
  for (const void* q : ptrs)
    if (!on_device(q)) return ADORYM_EINVAL;
  const int grads = (g_delta ? 1 : 0) | (g_probe ? 2 : 0) | (g_pos ? 4 : 0);
  Plan pl;
  const char* msg = "";
  int rc = make_plan(*p, true, grads, loss_out != nullptr, &pl, &msg);
  if (rc) return rc;
  // the staging areas of the plan are for host arguments, which this entry point does not take
  const size_t tab_off = (pl.off_s_probe + 255) & ~(size_t)255;
  const size_t ntab = table_count(*p);
  if (tab_off + ntab * sizeof(float2) > kScratchBytes) return ADORYM_ETOOBIG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return ADORYM_EDEVICE;
  }
  char* ws = nullptr;
  if ((rc = scratch_address(dev, &ws))) return rc;
  if ((rc = prepare_kernels(*p, &msg))) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  // tables: twiddles, two propagator factors and up to four detector factors, built on the device
  {
    const int n = (int)ntab, nt = 256;
    const double* nf = p->nf;
    k_noalloc_tables<<<(n + nt - 1) / nt, nt, 0, s>>>(reinterpret_cast<float2*>(ws + tab_off), p->N,
                                                       p->lambda_dz_over_px2, p->farfield ? 0 : p->n_dist, nf[0],
                                                       nf[1], nf[2], nf[3]);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return ADORYM_EDEVICE;
  }
  Tables t;
  t.dev = reinterpret_cast<float2*>(ws + tab_off);
  t.N = p->N;
  t.nd = p->farfield ? 0 : p->n_dist;
  Object obj;
  obj.d = delta;
  obj.b = beta;
  obj.Lz = p->Lz;
  obj.Ly = p->Ly;
  obj.Lx = p->Lx;
  CallPtrs c;
  c.probe = reinterpret_cast<const float2*>(probe);
  c.pos = pos;
  c.I_meas = I_meas;
  c.loss = loss_out;
  c.gd = g_delta;
  c.gb = g_beta;
  c.g_probe = reinterpret_cast<float2*>(g_probe);
  c.g_pos = g_pos;
  c.I_out = I_out;
  c.status = status;   // caller-zeroed device word; null: the scratch word, cleared on the stream
  std::string err;
  rc = enqueue(pl, obj, t, c, ws, s, &err);
  if (rc) return rc;
  if (cudaGetLastError() != cudaSuccess) return ADORYM_EDEVICE;
  return ADORYM_OK;
}
