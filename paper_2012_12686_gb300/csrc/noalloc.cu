// adorym_loss_grad_noalloc: the loss/gradient call for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a CUDA stream capture they do
// not control, plug-ins of host frameworks that own every device allocation through their own
// pool, or real-time loops where an allocation (and the device synchronisation it can bring) is
// not acceptable.  This entry point therefore draws all of its workspace -- checkpoints,
// segment buffers, far-field and loss partials, probe-gradient partials and the FP64-built
// twiddle/propagator tables -- from one file-scope device array of fixed size, and calls no
// cudaMalloc, cudaFree or other allocating routine.  The caller still passes every input and
// output, as device pointers.
//
// The array (ADORYM_NOALLOC_SCRATCH_BYTES) is reserved on every GPU that loads this code and
// stays reserved until the process exits.  Its device address is looked up once per device with
// cudaGetSymbolAddress (the name is only a host-side stand-in for the device address), on the
// first call made with that device current -- so make the first call on a device before any
// stream capture.  All calls share the array and it keeps the last call's contents: the parts
// that must start at zero are cleared on the stream by each call, and calls whose work overlaps
// on the GPU (different streams, or several host threads) race on it and must be serialised by
// the caller.
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

}  // namespace

using namespace adorym;

extern "C" int adorym_loss_grad_noalloc(void* cuda_stream, const adorym_problem* p, const float* delta,
                                        const float* beta, const float* probe, const float* pos,
                                        const float* I_meas, double* loss_out, float* g_delta, float* g_beta,
                                        float* g_probe, float* g_pos, float* I_out) {
  if (!p || !delta || !beta || !probe || !pos || !I_meas) return ADORYM_EINVAL;
  if (p->gaps && p->L > 1) return ADORYM_EINVAL;   // per-gap tables would not fit the fixed host buffer
  if ((g_delta == nullptr) != (g_beta == nullptr)) return ADORYM_EINVAL;
  const void* ptrs[] = {delta, beta, probe, pos, I_meas, loss_out, g_delta, g_beta, g_probe, g_pos, I_out};
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
  // tables are built on the host stack and copied into the scratch: twiddles, two propagator
  // factors and up to four detector factors of N <= 1024 values each
  constexpr size_t kTab = 7 * 1024;
  if (ntab > kTab) return ADORYM_EINVAL;
  float2 tab[kTab];
  fill_tables(*p, tab);
  if (cudaMemcpyAsync(ws + tab_off, tab, ntab * sizeof(float2), cudaMemcpyHostToDevice, s) != cudaSuccess) {
    cudaGetLastError();
    return ADORYM_EDEVICE;
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
  std::string err;
  rc = enqueue(pl, obj, t, c, ws, s, &err);
  if (rc) return rc;
  if (cudaGetLastError() != cudaSuccess) return ADORYM_EDEVICE;
  return ADORYM_OK;
}
