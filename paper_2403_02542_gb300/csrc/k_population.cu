// Population control by comb resampling.  The paper does not describe a
// population-control scheme; the reading taken here is the comb with a
// caller-supplied uniform u: with cumulative weights C_w = W_0 + ... + W_w
// summed in walker order in FP64, tooth j at (u + j) C_{Nw-1} / Nw selects the
// first walker w with C_w > tooth.  Every slot then holds a copy of its
// selected walker with weight C_{Nw-1} / Nw (total weight kept).
#include "internal.cuh"

namespace afq {

namespace {

// One block: sequential cumulative sum (thread 0), then one binary search per tooth.
__global__ void __launch_bounds__(1024) comb_kernel(const double* __restrict__ weight, double* __restrict__ cum,
                                                    int* __restrict__ idx, int* __restrict__ index_out,
                                                    double* __restrict__ total_out, int Nw, double u) {
  __shared__ double s_total;
  if (threadIdx.x == 0) {
    double acc = 0.0;
    for (int w = 0; w < Nw; ++w) {
      acc = acc + weight[w];
      cum[w] = acc;
    }
    s_total = acc;
    *total_out = acc;
  }
  __syncthreads();
  const double total = s_total;
  const bool ok = total > 0.0 && isfinite(total);
  for (int j = threadIdx.x; j < Nw; j += blockDim.x) {
    int pick = -1;
    if (ok) {
      const double tooth = (u + (double)j) * total / (double)Nw;
      int lo = 0, hi = Nw - 1;  // first w with cum[w] > tooth, clamped to Nw - 1
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (tooth < cum[mid]) hi = mid; else lo = mid + 1;
      }
      pick = lo;
    }
    idx[j] = pick;
    if (index_out) index_out[j] = pick;
  }
}

template <typename R>
__global__ void comb_gather_kernel(const typename C2<R>::t* __restrict__ psi, typename C2<R>::t* __restrict__ out,
                                   const int* __restrict__ idx, size_t per, int Nw) {
  const size_t total = per * Nw;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / per);
    const int src = idx[j];
    out[e] = psi[(size_t)(src < 0 ? j : src) * per + e % per];
  }
}

template <typename R>
__global__ void comb_scatter_kernel(typename C2<R>::t* __restrict__ psi, const typename C2<R>::t* __restrict__ in,
                                    double* __restrict__ weight, double* __restrict__ logovl, uint32_t* __restrict__ status,
                                    const double* __restrict__ lo_tmp, const uint32_t* __restrict__ st_tmp,
                                    const int* __restrict__ idx, const double* __restrict__ total, size_t per, int Nw) {
  const size_t all = per * Nw;
  const bool ok = idx[0] >= 0;  // the comb ran (positive, finite total weight)
  if (!ok) return;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < all; e += (size_t)gridDim.x * blockDim.x) {
    psi[e] = in[e];
    if (e % per == 0) {
      const int j = (int)(e / per);
      weight[j] = *total / (double)Nw;
      logovl[2 * j] = lo_tmp[2 * j];
      logovl[2 * j + 1] = lo_tmp[2 * j + 1];
      status[j] = st_tmp[j];
    }
  }
}

__global__ void comb_side_kernel(const double* __restrict__ logovl, const uint32_t* __restrict__ status,
                                 double* __restrict__ lo_tmp, uint32_t* __restrict__ st_tmp, const int* __restrict__ idx,
                                 int Nw) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= Nw) return;
  const int src = idx[j] < 0 ? j : idx[j];
  lo_tmp[2 * j] = logovl[2 * src];
  lo_tmp[2 * j + 1] = logovl[2 * src + 1];
  st_tmp[j] = status[src];
}

inline int grid_for(size_t n) {
  size_t b = (n + 255) / 256;
  return (int)(b > 152 * 32 ? 152 * 32 : (b == 0 ? 1 : b));
}

}  // namespace

template <typename R>
cudaError_t launch_comb(afqmc_ctx* c, const afqmc_walkers* w, double u, int* index_out, cudaStream_t s) {
  Workspace& ws = c->ws;
  const int Nw = w->n_walkers;
  const size_t per = (size_t)c->nc * c->N;
  double* cum = ws.epart;                             // [Nw]
  int* idx = reinterpret_cast<int*>(ws.scal);         // [Nw]
  double* total = ws.emix;                            // [1]
  double* lo_tmp = ws.eloc;                           // [Nw][2]
  uint32_t* st_tmp = reinterpret_cast<uint32_t*>(ws.ecap);  // [Nw]
  comb_kernel<<<1, 1024, 0, s>>>(w->weight, cum, idx, index_out, total, Nw, u);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  comb_gather_kernel<R><<<grid_for(per * Nw), 256, 0, s>>>(static_cast<const typename C2<R>::t*>(w->psi),
                                                          static_cast<typename C2<R>::t*>(ws.psi_new), idx, per, Nw);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  comb_side_kernel<<<(Nw + 255) / 256, 256, 0, s>>>(w->logovl, w->status, lo_tmp, st_tmp, idx, Nw);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  comb_scatter_kernel<R><<<grid_for(per * Nw), 256, 0, s>>>(static_cast<typename C2<R>::t*>(w->psi),
                                                           static_cast<const typename C2<R>::t*>(ws.psi_new),
                                                           w->weight, w->logovl, w->status, lo_tmp, st_tmp, idx,
                                                           total, per, Nw);
  return cudaGetLastError();
}

template cudaError_t launch_comb<double>(afqmc_ctx*, const afqmc_walkers*, double, int*, cudaStream_t);
template cudaError_t launch_comb<float>(afqmc_ctx*, const afqmc_walkers*, double, int*, cudaStream_t);

}  // namespace afq
