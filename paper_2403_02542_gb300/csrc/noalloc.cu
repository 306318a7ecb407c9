// afqmc_local_energy_static: the local-energy entry point for callers that
// must not allocate device memory.
//
// Some callers cannot call cudaMalloc when they need an energy: code that
// runs while a framework's caching allocator owns the whole device, code
// with a hard memory budget fixed at start-up, or code that must not
// synchronise the device (cudaMalloc/cudaFree may do so).  The ordinary
// afqmc_local_energy grows the context's workspace with cudaMalloc when the
// walker count rises; this variant instead carves its scratch (Theta, the
// log-determinants, per-walker scalars, the per-(walker, g) partial sums and
// the capped energies) out of one file-scope __device__ array of fixed size,
// which the CUDA runtime reserves on every device that loads this library
// and keeps until the process exits.  It runs exactly the kernels of
// afqmc_local_energy.
#include <cmath>
#include <mutex>

#include "internal.cuh"

namespace {

constexpr size_t kScratchBytes = AFQMC_STATIC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};  // device address per device ordinal
std::mutex g_scratch_mu;

inline size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

using namespace afq;

extern "C" afqmc_status afqmc_local_energy_static(afqmc_ctx* c, const afqmc_walkers* w, double e0, double tau,
                                                  double* e_loc, double* e_mix) {
  if (!c || !w || !e_loc || !e_mix) return AFQMC_EINVAL;
  if (w->n_walkers < 0 || (w->n_walkers > 0 && (!w->psi || !w->weight || !w->logovl || !w->status)))
    return AFQMC_EINVAL;
  const size_t align = c->prec == AFQMC_FP64 ? 16 : 8;
  if (((uintptr_t)w->psi) % align || ((uintptr_t)w->weight) % 8 || ((uintptr_t)e_loc) % 8 ||
      ((uintptr_t)e_mix) % 8 || ((uintptr_t)w->status) % 4)
    return AFQMC_EINVAL;
  if (!std::isfinite(tau) || !std::isfinite(e0)) return AFQMC_EDOM;
  if (!(tau > 0.0)) return AFQMC_EINVAL;
  if (w->n_walkers == 0) return AFQMC_OK;

  // scratch layout; every slice starts on a 256-byte boundary
  const size_t Nw = (size_t)w->n_walkers;
  const size_t cs = c->prec == AFQMC_FP64 ? 16 : 8;
  const size_t b_theta = up256(Nw * c->nc * c->N * cs);
  const size_t b_logdet = up256(Nw * 4 * sizeof(double));
  const size_t b_scal = up256(Nw * SC_COUNT * sizeof(double));
  const size_t b_epart = up256(Nw * (size_t)c->G * 8 * sizeof(double));
  const size_t b_ecap = up256(Nw * sizeof(double));
  // split Theta planes of the tensor-core exchange (mixed contexts that use it)
  const size_t b_plane = c->tc.ok ? up256(tc_exchange_plane_bytes(c->tc, w->n_walkers)) : 0;
  const size_t need = b_theta + b_logdet + b_scal + b_epart + b_ecap + 2 * b_plane;
  if (need > kScratchBytes) return AFQMC_EINVAL;  // beyond AFQMC_STATIC_SCRATCH_BYTES

  // device address of the array on the current device, resolved once per device.
  // The context's memory and stream belong to the device that was current at
  // afqmc_create; the array's address is per device, so a call from another
  // device is refused before anything is launched.
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return AFQMC_ECUDA;
  if (dev != c->device) return AFQMC_EINVAL;
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return AFQMC_ECUDA;
      g_scratch_addr[dev] = p;
    }
    base = g_scratch_addr[dev];
  }

  // a shallow copy of the context whose workspace points into the array
  afqmc_ctx tmp = *c;
  tmp.prof.on = false;
  char* p = static_cast<char*>(base);
  tmp.ws.theta = p;
  p += b_theta;
  tmp.ws.logdet = reinterpret_cast<double*>(p);
  p += b_logdet;
  tmp.ws.scal = reinterpret_cast<double*>(p);
  p += b_scal;
  tmp.ws.epart = reinterpret_cast<double*>(p);
  p += b_epart;
  tmp.ws.ecap = reinterpret_cast<double*>(p);
  p += b_ecap;
  if (c->tc.ok) {  // same tensor-core kernels, operand planes in the array (maps are host-side)
    void* hi = p;
    void* lo = p + b_plane;
    if (tc_exchange_bind(tmp.tc, hi, lo, w->n_walkers) != cudaSuccess) return AFQMC_ECUDA;
  }

  cudaStream_t s = c->stream;
  int nl = 0;
  cudaError_t e;
  if (c->prec == AFQMC_FP64) {
    e = launch_overlap<double>(&tmp, w->n_walkers, w->psi, tmp.ws.theta, tmp.ws.logdet, w->status, s);
    if (e == cudaSuccess) e = launch_energy<double>(&tmp, w->n_walkers, w->weight, e0, tau, e_loc, e_mix, s, &nl);
  } else {
    e = launch_overlap<float>(&tmp, w->n_walkers, w->psi, tmp.ws.theta, tmp.ws.logdet, w->status, s);
    if (e == cudaSuccess) e = launch_energy<float>(&tmp, w->n_walkers, w->weight, e0, tau, e_loc, e_mix, s, &nl);
  }
  c->launches += 1 + nl;
  return e == cudaSuccess ? AFQMC_OK : AFQMC_ECUDA;
}
