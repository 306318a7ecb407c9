// Block-Krylov action of the exponential (Sec. IV.D, Eqs. bkrylovsub-bkrylov)
// for every walker and spin block: Psi_s = B_1 R (QR), the orthonormal basis
// B_k = [B_1 .. B_k] of span{Psi_s, A Psi_s, .., A^{k-1} Psi_s} by block
// Arnoldi, the block upper Hessenberg A_k = B_k^dagger A B_k, and
// bkrylov_k = B_k e^{A_k} E_n R.
//
// Readings (the paper leaves them open): the QR of Psi_s and of every new
// block is modified Gram-Schmidt; a new block is orthogonalised against the
// previous ones by one block modified Gram-Schmidt pass; at most N / n blocks;
// the space is invariant at the first new block whose QR has a diagonal
// entry <= 1e-12 ||A||_F.  e^{A_k} E_n is the Taylor series of e^{A_k / s}
// applied s times (s = ceil ||A_k||_1 / 4), each series summed until its
// terms fall below the working precision.
//
// One block of 128 threads per (walker, spin); the basis blocks live in the
// Krylov basis slots of the workspace ([slot][w][na+nb][N], the spin's
// columns), the products A B_j are the step's walker-batched A V products.
// Walker states, the basis and A_k are in the walkers' precision; norms and
// the series' convergence tests are FP64.
#include "internal.cuh"

namespace afq {

namespace {

constexpr int BKT = 128;  // threads per (walker, spin) block

template <typename R>
struct cz {
  R re, im;
};
template <typename R>
__device__ __forceinline__ cz<R> operator+(cz<R> a, cz<R> b) { return cz<R>{a.re + b.re, a.im + b.im}; }
template <typename R>
__device__ __forceinline__ cz<R> operator-(cz<R> a, cz<R> b) { return cz<R>{a.re - b.re, a.im - b.im}; }
template <typename R>
__device__ __forceinline__ cz<R> operator*(cz<R> a, cz<R> b) {
  return cz<R>{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ cz<R> cjmul(cz<R> a, cz<R> b) {  // conj(a) b
  return cz<R>{a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <typename R>
__device__ __forceinline__ cz<R> ld(const typename C2<R>::t& v) { return cz<R>{v.x, v.y}; }
template <typename R>
__device__ __forceinline__ typename C2<R>::t st(cz<R> v) {
  typename C2<R>::t o;
  o.x = v.re;
  o.y = v.im;
  return o;
}

template <typename R>
__device__ __forceinline__ R wsum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum (or maximum) of one double per thread over the block, fixed order.
__device__ double block_reduce(double v, bool take_max, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double u = __shfl_xor_sync(0xffffffffu, v, o);
    v = take_max ? fmax(v, u) : v + u;
  }
  __syncthreads();  // the previous use of sh is over
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = sh[0];
  for (int i = 1; i < (int)(blockDim.x >> 5); ++i) t = take_max ? fmax(t, sh[i]) : t + sh[i];
  return t;
}

// Per (walker, spin) area of the block-Krylov workspace, in complex elements
// of the walkers' type: A_k [M][M] (row-major), R [nm][nm], F [M][nm], with
// M = k * nm, nm = max(na, nb).
struct BkLayout {
  size_t M, nm, stride;
  __host__ __device__ BkLayout(int k, int nmax) {
    M = (size_t)k * nmax;
    nm = (size_t)nmax;
    stride = M * M + nm * nm + M * nm;
  }
};

// Modified Gram-Schmidt QR of the n columns X[b][p] (shared memory, column b
// at X + b * XS) in place, right-looking: once q_j is final every later column
// is projected on it, so each column receives the projections q_0, q_1, ...
// in order.  R[j][l] is written to Rg (row stride ld).  Returns false when a
// diagonal entry is <= tol (the columns are then left finite).
template <typename R>
__device__ bool mgs_smem(cz<R>* X, int N, int XS, int n, typename C2<R>::t* Rg, int ld, double tol, double* sh) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  __shared__ R s_inv;
  bool ok = true;
  for (int j = 0; j < n; ++j) {
    cz<R>* xj = X + (size_t)j * XS;
    double part = 0.0;
    for (int p = tid; p < N; p += blockDim.x) part += (double)xj[p].re * xj[p].re + (double)xj[p].im * xj[p].im;
    const double r = sqrt(block_reduce(part, false, sh));
    const bool good = r > tol && isfinite(r);
    ok = ok && good;
    if (tid == 0) {
      s_inv = good ? (R)(1.0 / r) : R(0);
      Rg[(size_t)j * ld + j] = st(cz<R>{good ? (R)r : R(0), R(0)});
    }
    __syncthreads();
    const R inv = s_inv;
    for (int p = tid; p < N; p += blockDim.x) xj[p] = cz<R>{xj[p].re * inv, xj[p].im * inv};
    for (int l = tid; l < j; l += blockDim.x) Rg[(size_t)j * ld + l] = st(cz<R>{R(0), R(0)});
    __syncthreads();
    for (int l = j + 1 + wid; l < n; l += nw) {  // one warp per later column
      cz<R>* xl = X + (size_t)l * XS;
      R dr = R(0), di = R(0);
      for (int p = lane; p < N; p += 32) {
        const cz<R> d = cjmul(xj[p], xl[p]);
        dr += d.re;
        di += d.im;
      }
      dr = wsum(dr);
      di = wsum(di);
      if (lane == 0) Rg[(size_t)j * ld + l] = st(cz<R>{dr, di});
      const cz<R> h{dr, di};
      for (int p = lane; p < N; p += 32) xl[p] = xl[p] - h * xj[p];
    }
    __syncthreads();
  }
  return ok;
}

// QR of the spin block of psi_b into basis slot 0 and R; A_k zeroed;
// k_eff = min(k, N / n).
template <typename R>
__global__ void __launch_bounds__(BKT) bk_start_kernel(const typename C2<R>::t* __restrict__ X,
                                                        typename C2<R>::t* __restrict__ basis,
                                                        typename C2<R>::t* __restrict__ bk, int* __restrict__ keff,
                                                        int N, int na, int nb, int kl, int k) {
  typedef typename C2<R>::t P;
  extern __shared__ double bk_smem[];
  __shared__ double sh[BKT / 32];
  const int w = blockIdx.x, spin = blockIdx.y;
  const int n = spin ? nb : na, off = spin ? na : 0, nc = na + nb;
  const int nmax = na > nb ? na : nb;
  if (n == 0) return;
  const BkLayout L(kl, nmax);  // area layout for kl blocks (k <= kl requested)
  P* area = bk + ((size_t)w * 2 + spin) * L.stride;
  for (size_t e = threadIdx.x; e < L.M * L.M; e += blockDim.x) area[e] = st(cz<R>{R(0), R(0)});
  cz<R>* Xs = reinterpret_cast<cz<R>*>(bk_smem);
  const P* src = X + ((size_t)w * nc + off) * N;
  for (int e = threadIdx.x; e < n * N; e += blockDim.x) Xs[e] = ld<R>(src[e]);
  __syncthreads();
  mgs_smem<R>(Xs, N, N, n, area + L.M * L.M, (int)L.nm, 0.0, sh);
  P* dst = basis + ((size_t)w * nc + off) * N;
  for (int e = threadIdx.x; e < n * N; e += blockDim.x) dst[e] = st(Xs[e]);
  if (threadIdx.x == 0) {
    const int ks = N / n < k ? N / n : k;
    keff[w * 2 + spin] = ks > 0 ? ks : 1;
  }
}

// Block j of the Arnoldi process: W = A B_j (in W) is orthogonalised against
// B_0 .. B_j (block MGS, A_k blocks (i, j)), then B_{j+1} H_{j+1,j} = QR(W).
template <typename R>
__global__ void __launch_bounds__(BKT) bk_orth_kernel(const typename C2<R>::t* __restrict__ W,
                                                       typename C2<R>::t* __restrict__ basis, size_t bstride,
                                                       typename C2<R>::t* __restrict__ bk, int* __restrict__ keff,
                                                       const double* __restrict__ scal, int N, int na, int nb,
                                                       int k, int j) {
  typedef typename C2<R>::t P;
  extern __shared__ double bk_smem[];
  __shared__ double sh[BKT / 32];
  const int w = blockIdx.x, spin = blockIdx.y;
  const int n = spin ? nb : na, off = spin ? na : 0, nc = na + nb;
  const int nmax = na > nb ? na : nb;
  if (n == 0 || keff[w * 2 + spin] <= j) return;
  const int tid = threadIdx.x;
  const BkLayout L(k, nmax);
  P* H = bk + ((size_t)w * 2 + spin) * L.stride;
  // W and B_i staged with row stride N + 1 (the entry loop reads them across
  // rows: the odd stride spreads the rows over the banks)
  const int NS = N + 1;
  cz<R>* Ws = reinterpret_cast<cz<R>*>(bk_smem);  // [n][NS]
  cz<R>* Bs = Ws + (size_t)n * NS;                 // [n][NS]
  cz<R>* Hs = Bs + (size_t)n * NS;                 // [n][n]
  const size_t col0 = (size_t)w * nc + off;
  for (int e = tid; e < n * N; e += blockDim.x) {
    const int b = e / N, p = e - (e / N) * N;
    Ws[b * NS + p] = ld<R>(W[col0 * N + e]);
  }
  for (int i = 0; i <= j; ++i) {
    const P* Bi = basis + (size_t)i * bstride + col0 * N;
    for (int e = tid; e < n * N; e += blockDim.x) {
      const int a = e / N, p = e - (e / N) * N;
      Bs[a * NS + p] = ld<R>(Bi[e]);
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += blockDim.x) {  // H_ij[a][b] = B_i[:, a]^dagger W[:, b]
      const int a = e / n, b = e - (e / n) * n;
      const cz<R>* x = Bs + (size_t)a * NS;
      const cz<R>* y = Ws + (size_t)b * NS;
      cz<R> acc{R(0), R(0)};
      for (int p = 0; p < N; ++p) acc = acc + cjmul(x[p], y[p]);
      Hs[e] = acc;
      H[((size_t)i * n + a) * L.M + (size_t)j * n + b] = st(acc);
    }
    __syncthreads();
    for (int e = tid; e < n * N; e += blockDim.x) {  // W -= B_i H_ij
      const int b = e / N, p = e - (e / N) * N;
      cz<R> acc{R(0), R(0)};
      for (int a = 0; a < n; ++a) acc = acc + Bs[a * NS + p] * Hs[a * n + b];
      Ws[b * NS + p] = Ws[b * NS + p] - acc;
    }
    __syncthreads();
  }
  if (j + 1 >= keff[w * 2 + spin]) return;
  // B_{j+1} H_{j+1,j} = QR(W); R into the subdiagonal block of A_k
  const double tol = 1e-12 * scal[(size_t)w * SC_COUNT + SC_NORMA];
  const bool ok = mgs_smem<R>(Ws, N, NS, n, H + ((size_t)(j + 1) * n) * L.M + (size_t)j * n, (int)L.M, tol, sh);
  P* dst = basis + (size_t)(j + 1) * bstride + col0 * N;
  if (ok) {
    for (int e = tid; e < n * N; e += blockDim.x) {
      const int b = e / N, p = e - (e / N) * N;
      dst[e] = st(Ws[b * NS + p]);
    }
  } else {
    // invariant subspace: stop here; the slot stays finite for the next product
    for (int e = tid; e < n * N; e += blockDim.x) dst[e] = st(cz<R>{R(0), R(0)});
    for (int e = tid; e < n * n; e += blockDim.x) {
      const int a = e / n, b = e - (e / n) * n;
      H[((size_t)(j + 1) * n + a) * L.M + (size_t)j * n + b] = st(cz<R>{R(0), R(0)});
    }
    if (tid == 0) keff[w * 2 + spin] = j + 1;
  }
}

// F = e^{A_k} E_n R for the k_eff n leading rows and columns of A_k.
template <typename R>
__global__ void __launch_bounds__(BKT) bk_expm_kernel(typename C2<R>::t* __restrict__ bk,
                                                       const int* __restrict__ keff, int na, int nb, int k) {
  typedef typename C2<R>::t P;
  extern __shared__ double bk_smem[];
  __shared__ double sh[BKT / 32];
  const int w = blockIdx.x, spin = blockIdx.y;
  const int n = spin ? nb : na;
  const int nmax = na > nb ? na : nb;
  if (n == 0) return;
  const int tid = threadIdx.x;
  const BkLayout L(k, nmax);
  P* area = bk + ((size_t)w * 2 + spin) * L.stride;
  const int m = keff[w * 2 + spin] * n;
  // A_k column-major in shared memory (Hs[c * m + r] = A_k[r][c]): the lanes
  // of a warp take consecutive rows r of one product column, so they read
  // consecutive words
  cz<R>* Hs = reinterpret_cast<cz<R>*>(bk_smem);
  cz<R>* X = Hs + (size_t)m * m;                   // [n][m]: column b of the running result
  cz<R>* T = X + (size_t)m * n;                    // current series term
  cz<R>* U = T + (size_t)m * n;                    // next term
  for (int e = tid; e < m * m; e += blockDim.x) {
    const int r = e / m, c = e - (e / m) * m;
    Hs[(size_t)c * m + r] = ld<R>(area[(size_t)r * L.M + c]);
  }
  for (int e = tid; e < m * n; e += blockDim.x) {
    const int b = e / m, r = e - (e / m) * m;
    X[e] = cz<R>{r == b ? R(1) : R(0), R(0)};
  }
  double cs = 0.0;  // ||A_k||_1: largest column sum of |entries| (rows read along c)
  for (int c = tid; c < m; c += blockDim.x) {
    double t = 0.0;
    for (int r = 0; r < m; ++r) {
      const cz<R> h = ld<R>(area[(size_t)r * L.M + c]);
      t += sqrt((double)h.re * h.re + (double)h.im * h.im);
    }
    cs = fmax(cs, t);
  }
  const double norm1 = block_reduce(cs, true, sh);  // (its barriers also publish Hs and X)
  // sub-steps of norm <= 4: the terms peak near 4^4/4! ~ 11 before they fall,
  // a digit of headroom (bounded: a non-finite or huge norm takes at most 4096
  // sub-steps)
  const int nsteps = norm1 > 4.0 ? (norm1 < 16384.0 ? (int)ceil(0.25 * norm1) : 4096) : 1;
  const double eps = std::is_same<R, double>::value ? 1.1e-16 : 6.0e-8;
  const int max_terms = std::is_same<R, double>::value ? 40 : 24;
  for (int step = 0; step < nsteps; ++step) {
    for (int e = tid; e < m * n; e += blockDim.x) T[e] = X[e];
    __syncthreads();
    for (int t = 1; t <= max_terms; ++t) {
      const R scale = (R)(1.0 / ((double)nsteps * t));
      double tmax = 0.0, xmax = 0.0;
      for (int e = tid; e < m * n; e += blockDim.x) {  // U = A_k T / (s t); X += U
        const int b = e / m, r = e - (e / m) * m;
        const cz<R>* tb = T + (size_t)b * m;
        cz<R> acc{R(0), R(0)};
        for (int c = 0; c < m; ++c) acc = acc + Hs[(size_t)c * m + r] * tb[c];
        acc = cz<R>{acc.re * scale, acc.im * scale};
        U[e] = acc;
        const cz<R> x = X[e] + acc;
        X[e] = x;
        tmax = fmax(tmax, fabs((double)acc.re) + fabs((double)acc.im));
        xmax = fmax(xmax, fabs((double)x.re) + fabs((double)x.im));
      }
      const double tm = block_reduce(tmax, true, sh);
      const double xm = block_reduce(xmax, true, sh);  // (its barriers also order U before the swap)
      cz<R>* tmp = T;
      T = U;
      U = tmp;
      if (tm <= eps * xm) break;
    }
    __syncthreads();
  }
  // F = X R (R upper triangular, n x n), rows r < m, columns b < n
  const P* Rg = area + L.M * L.M;
  P* F = area + L.M * L.M + L.nm * L.nm;
  for (int e = tid; e < m * n; e += blockDim.x) {
    const int r = e / n, b = e - (e / n) * n;
    cz<R> acc{R(0), R(0)};
    for (int a = 0; a <= b; ++a) acc = acc + X[(size_t)a * m + r] * ld<R>(Rg[(size_t)a * L.nm + b]);
    F[(size_t)r * L.nm + b] = st(acc);
  }
}

// out[:, spin columns] = sum_{i < k_eff} B_i F_i (F_i: rows i n .. i n + n - 1 of F).
template <typename R>
__global__ void __launch_bounds__(BKT) bk_combine_kernel(const typename C2<R>::t* __restrict__ basis, size_t bstride,
                                                          const typename C2<R>::t* __restrict__ bk,
                                                          const int* __restrict__ keff,
                                                          typename C2<R>::t* __restrict__ out, int N, int na, int nb,
                                                          int k) {
  typedef typename C2<R>::t P;
  extern __shared__ double bk_smem[];
  const int w = blockIdx.x, spin = blockIdx.y;
  const int n = spin ? nb : na, off = spin ? na : 0, nc = na + nb;
  const int nmax = na > nb ? na : nb;
  if (n == 0) return;
  const BkLayout L(k, nmax);
  const int ke = keff[w * 2 + spin], m = ke * n;
  const P* F = bk + ((size_t)w * 2 + spin) * L.stride + L.M * L.M + L.nm * L.nm;
  cz<R>* Fs = reinterpret_cast<cz<R>*>(bk_smem);  // [m][n]
  for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
    const int r = e / n, b = e - (e / n) * n;
    Fs[e] = ld<R>(F[(size_t)r * L.nm + b]);
  }
  __syncthreads();
  const size_t col0 = (size_t)w * nc + off;
  cz<R>* Bs = Fs + (size_t)m * n;  // [m][N]: the k_eff basis blocks stacked, row i n + a = B_i[:, a]
  for (int i = 0; i < ke; ++i) {
    const P* Bi = basis + (size_t)i * bstride + col0 * N;
    for (int e = threadIdx.x; e < n * N; e += blockDim.x) Bs[(size_t)i * n * N + e] = ld<R>(Bi[e]);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * N; e += blockDim.x) {
    const int b = e / N, p = e - (e / N) * N;
    cz<R> acc{R(0), R(0)};
    for (int r = 0; r < m; ++r) acc = acc + Bs[(size_t)r * N + p] * Fs[r * n + b];
    out[col0 * N + e] = st(acc);
  }
}

template <typename F>
cudaError_t bk_smem_limit(const afqmc_ctx* c, F* f, size_t bytes) {
  if (capturing(c) || bytes <= 48 * 1024) return cudaSuccess;
  return raise_smem_limit(f);
}

}  // namespace

// shared-memory bytes of the small-exponential and the Arnoldi kernels
size_t bk_expm_smem(int k, int nmax, size_t csize) {
  const size_t m = (size_t)k * nmax;
  return (m * m + 3 * m * nmax) * csize;
}
size_t bk_combine_smem(int N, int k, int nmax, size_t csize) {
  return (size_t)k * nmax * ((size_t)nmax + N) * csize;
}
size_t bk_orth_smem(int N, int nmax, size_t csize) {
  return (2 * (size_t)nmax * (N + 1) + (size_t)nmax * nmax) * csize;
}

cudaError_t bk_ensure(afqmc_ctx* c, int Nw, int k) {
  Workspace& ws = c->ws;
  const int nmax = c->na > c->nb ? c->na : c->nb;
  if (ws.bk && Nw <= ws.bk_cap && k <= ws.bk_k) return cudaSuccess;
  const int cap = Nw > ws.bk_cap ? Nw : ws.bk_cap;
  const int kk = k > ws.bk_k ? k : ws.bk_k;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return e;
  if (ws.bk) cudaFree(ws.bk);
  if (ws.bk_keff) cudaFree(ws.bk_keff);
  ws.bk = nullptr;
  ws.bk_keff = nullptr;
  ws.bk_cap = ws.bk_k = 0;
  const size_t cs = c->prec == AFQMC_FP64 ? 16 : 8;
  const BkLayout L(kk, nmax);
  e = dmalloc(&ws.bk, (size_t)cap * 2 * L.stride * cs);
  if (e != cudaSuccess) return e;
  e = dmalloc(&ws.bk_keff, (size_t)cap * 2 * sizeof(int));
  if (e != cudaSuccess) return e;
  ws.bk_cap = cap;
  ws.bk_k = kk;
  return cudaSuccess;
}

template <typename R>
cudaError_t launch_bk_start(const afqmc_ctx* c, int Nw, int k, cudaStream_t s) {
  typedef typename C2<R>::t P;
  const int nmax = c->na > c->nb ? c->na : c->nb;
  const size_t shm = (size_t)nmax * c->N * sizeof(P);
  cudaError_t e = bk_smem_limit(c, bk_start_kernel<R>, shm);
  if (e != cudaSuccess) return e;
  bk_start_kernel<R><<<dim3(Nw, 2), BKT, shm, s>>>(static_cast<const P*>(c->ws.psi_b), static_cast<P*>(c->ws.basis),
                                                   static_cast<P*>(c->ws.bk), c->ws.bk_keff, c->N, c->na, c->nb,
                                                   c->ws.bk_k, k);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_bk_orth(const afqmc_ctx* c, int Nw, int j, cudaStream_t s) {
  typedef typename C2<R>::t P;
  const int nmax = c->na > c->nb ? c->na : c->nb;
  const size_t shm = bk_orth_smem(c->N, nmax, sizeof(P));
  cudaError_t e = bk_smem_limit(c, bk_orth_kernel<R>, shm);
  if (e != cudaSuccess) return e;
  const size_t bstride = (size_t)c->ws.n_walkers * c->nc * c->N;
  bk_orth_kernel<R><<<dim3(Nw, 2), BKT, shm, s>>>(static_cast<const P*>(c->ws.term0), static_cast<P*>(c->ws.basis),
                                                  bstride, static_cast<P*>(c->ws.bk), c->ws.bk_keff, c->ws.scal,
                                                  c->N, c->na, c->nb, c->ws.bk_k, j);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_bk_finish(const afqmc_ctx* c, int Nw, cudaStream_t s) {
  typedef typename C2<R>::t P;
  const int nmax = c->na > c->nb ? c->na : c->nb;
  const size_t shm = bk_expm_smem(c->ws.bk_k, nmax, sizeof(P));
  cudaError_t e = bk_smem_limit(c, bk_expm_kernel<R>, shm);
  if (e != cudaSuccess) return e;
  bk_expm_kernel<R><<<dim3(Nw, 2), BKT, shm, s>>>(static_cast<P*>(c->ws.bk), c->ws.bk_keff, c->na, c->nb,
                                                  c->ws.bk_k);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t shc = bk_combine_smem(c->N, c->ws.bk_k, nmax, sizeof(P));
  e = bk_smem_limit(c, bk_combine_kernel<R>, shc);
  if (e != cudaSuccess) return e;
  const size_t bstride = (size_t)c->ws.n_walkers * c->nc * c->N;
  bk_combine_kernel<R><<<dim3(Nw, 2), BKT, shc, s>>>(static_cast<const P*>(c->ws.basis), bstride,
                                                     static_cast<const P*>(c->ws.bk), c->ws.bk_keff,
                                                     static_cast<P*>(c->ws.acc), c->N, c->na, c->nb, c->ws.bk_k);
  return cudaGetLastError();
}

// kernel attributes before a graph capture
template <typename R>
cudaError_t prepare_bk(const afqmc_ctx*) {
  cudaError_t e = raise_smem_limit(bk_start_kernel<R>);
  if (e == cudaSuccess) e = raise_smem_limit(bk_orth_kernel<R>);
  if (e == cudaSuccess) e = raise_smem_limit(bk_expm_kernel<R>);
  if (e == cudaSuccess) e = raise_smem_limit(bk_combine_kernel<R>);
  return e;
}

#define AFQ_BK_INST(R)                                                                  \
  template cudaError_t launch_bk_start<R>(const afqmc_ctx*, int, int, cudaStream_t);    \
  template cudaError_t launch_bk_orth<R>(const afqmc_ctx*, int, int, cudaStream_t);     \
  template cudaError_t launch_bk_finish<R>(const afqmc_ctx*, int, cudaStream_t);        \
  template cudaError_t prepare_bk<R>(const afqmc_ctx*);
AFQ_BK_INST(double)
AFQ_BK_INST(float)
#undef AFQ_BK_INST

}  // namespace afq
