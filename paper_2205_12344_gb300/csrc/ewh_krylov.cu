// FP64 Krylov kernels for CG in the M inner product (Section 4.5, eq.
// amat_sym) and the conversions between the solver's dense vectors and the
// padded wave fields.  Reductions are deterministic: fixed per-thread strides,
// warp-shuffle and shared-memory trees of fixed shape, and a second pass that
// adds the per-block partial sums in a fixed order.
#include <cuda_runtime.h>

#include <string>

#include "ewh_internal.cuh"

namespace ewh {

constexpr int RED_THREADS = 256;

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double warp_part[RED_THREADS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) warp_part[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (wid == 0) {
    t = lane < RED_THREADS / 32 ? warp_part[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;  // valid in thread 0
}

// dense index -> (comp, node) decomposition helpers
__device__ __forceinline__ void node_coords(const Geom& g, long long node, int& x, int& y, int& z) {
  const long long nxy = (long long)g.nu[0] * g.nu[1];
  z = (int)(node / nxy);
  const long long r = node - (long long)z * nxy;
  y = (int)(r / g.nu[0]);
  x = (int)(r - (long long)y * g.nu[0]);
  x += g.off[0];
  y += g.off[1];
  z += g.off[2];
}

// The dense unknown layout [rhs][comp][z][y][x] walked by rows: block b takes
// rows b, b + gridDim.x, ... (row = ((rhs dim + comp) nu2 + z) nu1 + y), its
// threads the x of a row, so the index arithmetic is a few divisions per row
// and both the dense and the padded accesses are coalesced.  body(i, o, rhs):
// dense index i, padded offset o.
template <typename F>
__device__ __forceinline__ void for_dense_rows(const Geom& g, F body) {
  const int nu0 = g.nu[0], nu1 = g.nu[1], nu2 = g.nu[2];
  const long long nrows = (long long)g.nrhs * g.dim * nu2 * nu1;
  for (long long row = blockIdx.x; row < nrows; row += gridDim.x) {
    const int y = (int)(row % nu1);
    long long t = row / nu1;
    const int z = (int)(t % nu2);
    t /= nu2;
    const int comp = (int)(t % g.dim), rhs = (int)(t / g.dim);
    const long long i0 = row * nu0;
    const long long o0 = pidx(g, rhs, comp, g.off[0], y + g.off[1], z + g.off[2]);
    for (int x = threadIdx.x; x < nu0; x += blockDim.x) body(i0 + x, o0 + x, rhs);
  }
}

template <typename T>
__global__ void pack_kernel(Geom g, const double* __restrict__ dense, T* __restrict__ padded) {
  for_dense_rows(g, [&](long long i, long long o, int) { padded[o] = (T)dense[i]; });
}

template <typename T>
__global__ void unpack_kernel(Geom g, const T* __restrict__ padded, double* __restrict__ dense,
                              const double* __restrict__ sub_from) {
  for_dense_rows(g, [&](long long i, long long o, int) {
    const double v = (double)padded[o];
    dense[i] = sub_from ? sub_from[i] - v : v;
  });
}

template <typename T>
__global__ void pupdate_pack_kernel(Geom g, const double* __restrict__ r, double* __restrict__ p,
                                    const double* __restrict__ beta, T* __restrict__ padded) {
  for_dense_rows(g, [&](long long i, long long o, int rhs) {
    const double pn = r[i] + beta[rhs] * p[i];
    p[i] = pn;
    padded[o] = (T)pn;
  });
}

static int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

// launch shape of the row walks: one block per row (up to 16 per SM), a
// warp-multiple of threads up to 256
static dim3 rows_grid(const Geom& g) {
  long long rows = (long long)g.nrhs * g.dim * g.nu[2] * g.nu[1];
  if (rows > 152 * 16) rows = 152 * 16;
  return dim3((unsigned)(rows < 1 ? 1 : rows));
}
static dim3 rows_block(const Geom& g) {
  const int t = ((g.nu[0] + 31) / 32) * 32;
  return dim3(t > 256 ? 256 : t);
}

template <typename T>
cudaError_t launch_pack(const Geom& g, const double* dense, T* padded, cudaStream_t st) {
  pack_kernel<T><<<rows_grid(g), rows_block(g), 0, st>>>(g, dense, padded);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_unpack(const Geom& g, const T* padded, double* dense, const double* sub_from,
                          cudaStream_t st) {
  unpack_kernel<T><<<rows_grid(g), rows_block(g), 0, st>>>(g, padded, dense, sub_from);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_pupdate_pack(const Geom& g, const double* r, double* p, const double* beta, T* padded,
                                cudaStream_t st) {
  pupdate_pack_kernel<T><<<rows_grid(g), rows_block(g), 0, st>>>(g, r, p, beta, padded);
  return cudaGetLastError();
}

// ---- M inner products ------------------------------------------------------
int dot_blocks(const Geom& g) {
  const long long n = (long long)g.dim * g.nodes;
  long long b = (n + 4 * RED_THREADS - 1) / (4 * RED_THREADS);
  if (b > 1024) b = 1024;
  if (b < 1) b = 1;
  return (int)b;
}

// partial sums of sum_i mw[node(i)] x_i y_i over one rhs: grid (nblk, nrhs)
__global__ void mdot_partial_kernel(Geom g, const double* __restrict__ mw, const double* __restrict__ x,
                                    const double* __restrict__ y, double* __restrict__ part) {
  const int rhs = blockIdx.y;
  const long long n = (long long)g.dim * g.nodes;
  double s = 0.0;
  for (int c = 0; c < g.dim; ++c) {  // per component: the weight index is the node index
    const double* xr = x + (long long)rhs * n + (long long)c * g.nodes;
    const double* yr = y + (long long)rhs * n + (long long)c * g.nodes;
    for (long long j = blockIdx.x * (long long)RED_THREADS + threadIdx.x; j < g.nodes;
         j += (long long)gridDim.x * RED_THREADS)
      s += mw[j] * xr[j] * yr[j];
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[(long long)rhs * gridDim.x + blockIdx.x] = s;
}

__device__ double sum_partials(const double* part, int nblk) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += RED_THREADS) s += part[i];
  return block_sum(s);
}

__global__ void mdot_final_kernel(const double* __restrict__ part, int nblk, double* __restrict__ out) {
  const int rhs = blockIdx.x;
  const double s = sum_partials(part + (long long)rhs * nblk, nblk);
  if (threadIdx.x == 0) out[rhs] = s;
}

cudaError_t launch_mdot_partial(const Geom& g, const double* mw, const double* x, const double* y, double* part,
                                cudaStream_t st) {
  dim3 grd(dot_blocks(g), g.nrhs);
  mdot_partial_kernel<<<grd, RED_THREADS, 0, st>>>(g, mw, x, y, part);
  return cudaGetLastError();
}
cudaError_t launch_mdot_final(const Geom& g, const double* part, double* out, cudaStream_t st) {
  mdot_final_kernel<<<g.nrhs, RED_THREADS, 0, st>>>(part, dot_blocks(g), out);
  return cudaGetLastError();
}

// ---- CG scalar kernels -----------------------------------------------------
// flags bit 0: breakdown (pq <= 0 on an active rhs)
__global__ void cg_alpha_kernel(const double* __restrict__ pq_part, int nblk, const double* __restrict__ rr,
                                double* __restrict__ alpha, int* __restrict__ active, int* __restrict__ flags) {
  const int rhs = blockIdx.x;
  const double pq = sum_partials(pq_part + (long long)rhs * nblk, nblk);
  if (threadIdx.x == 0) {
    double a = 0.0;
    if (active[rhs]) {
      if (pq > 0.0 && isfinite(pq)) {
        a = rr[rhs] / pq;
      } else {
        atomicOr(flags, 1);
        active[rhs] = 0;
      }
    }
    alpha[rhs] = a;
  }
}

__global__ void cg_xr_kernel(Geom g, const double* __restrict__ mw, const double* __restrict__ alpha,
                             const double* __restrict__ p, const double* __restrict__ q, double* __restrict__ x,
                             double* __restrict__ r, double* __restrict__ part) {
  const int rhs = blockIdx.y;
  const long long n = (long long)g.dim * g.nodes;
  const double a = alpha[rhs];
  double s = 0.0;
  for (int c = 0; c < g.dim; ++c) {  // per component: the weight index is the node index
    const long long base = (long long)rhs * n + (long long)c * g.nodes;
    for (long long j = blockIdx.x * (long long)RED_THREADS + threadIdx.x; j < g.nodes;
         j += (long long)gridDim.x * RED_THREADS) {
      const long long k = base + j;
      x[k] += a * p[k];
      const double rn = r[k] - a * q[k];
      r[k] = rn;
      s += mw[j] * rn * rn;
    }
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[(long long)rhs * gridDim.x + blockIdx.x] = s;
}

__global__ void cg_beta_kernel(const double* __restrict__ part, int nblk, double* __restrict__ rr,
                               const double* __restrict__ bb, double* __restrict__ beta, double* __restrict__ res,
                               const int* __restrict__ active) {
  const int rhs = blockIdx.x;
  const double rn = sum_partials(part + (long long)rhs * nblk, nblk);
  if (threadIdx.x == 0) {
    if (active[rhs]) {
      beta[rhs] = rr[rhs] > 0.0 ? rn / rr[rhs] : 0.0;
      rr[rhs] = rn;
      res[rhs] = sqrt(rn / bb[rhs]);
    } else {
      beta[rhs] = 0.0;
    }
  }
}

// residual replacement: the recursive residual was overwritten by the true
// one with (r, r)_M = dot; rescale beta and reset rr accordingly
__global__ void cg_replace_kernel(int nrhs, const double* __restrict__ dot, double* __restrict__ rr,
                                  double* __restrict__ beta, double* __restrict__ res, const double* __restrict__ bb) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nrhs) return;
  beta[k] = rr[k] > 0.0 ? beta[k] * (dot[k] / rr[k]) : 0.0;
  rr[k] = dot[k];
  res[k] = sqrt(dot[k] / bb[k]);
}
cudaError_t launch_cg_replace(int nrhs, const double* dot, double* rr, double* beta, double* res, const double* bb,
                              cudaStream_t st) {
  cg_replace_kernel<<<(nrhs + 127) / 128, 128, 0, st>>>(nrhs, dot, rr, beta, res, bb);
  return cudaGetLastError();
}

// ---- conjugate residual pieces ---------------------------------------------
// res = sqrt((r, r)_M / bb) from the partial sums of (r, r)_M
__global__ void res_kernel(const double* __restrict__ part, int nblk, const double* __restrict__ bb,
                           double* __restrict__ res, const int* __restrict__ active) {
  const int rhs = blockIdx.x;
  const double rn = sum_partials(part + (long long)rhs * nblk, nblk);
  if (threadIdx.x == 0 && active[rhs]) res[rhs] = sqrt(rn / bb[rhs]);
}
// beta = (r, Ar)_new / (r, Ar)_old ; (r, Ar) = new   (sets it when init != 0)
__global__ void cr_beta_kernel(const double* __restrict__ part, int nblk, double* __restrict__ rar,
                               double* __restrict__ beta, const int* __restrict__ active, int init) {
  const int rhs = blockIdx.x;
  const double v = sum_partials(part + (long long)rhs * nblk, nblk);
  if (threadIdx.x == 0) {
    if (init) {
      rar[rhs] = v;
      beta[rhs] = 0.0;
    } else if (active[rhs]) {
      beta[rhs] = rar[rhs] != 0.0 ? v / rar[rhs] : 0.0;
      rar[rhs] = v;
    } else {
      beta[rhs] = 0.0;
    }
  }
}
// p = r + beta p ; Ap = Ar + beta Ap
__global__ void cr_pupdate_kernel(Geom g, const double* __restrict__ r, const double* __restrict__ ar,
                                  double* __restrict__ p, double* __restrict__ ap, const double* __restrict__ beta) {
  const long long n = (long long)g.dim * g.nodes;
  const long long total = n * g.nrhs;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const double b = beta[i / n];
    p[i] = r[i] + b * p[i];
    ap[i] = ar[i] + b * ap[i];
  }
}
cudaError_t launch_res(int nrhs, const double* part, int nblk, const double* bb, double* res, const int* active,
                       cudaStream_t st) {
  res_kernel<<<nrhs, RED_THREADS, 0, st>>>(part, nblk, bb, res, active);
  return cudaGetLastError();
}
cudaError_t launch_cr_beta(int nrhs, const double* part, int nblk, double* rar, double* beta, const int* active,
                           int init, cudaStream_t st) {
  cr_beta_kernel<<<nrhs, RED_THREADS, 0, st>>>(part, nblk, rar, beta, active, init);
  return cudaGetLastError();
}
cudaError_t launch_cr_pupdate(const Geom& g, const double* r, const double* ar, double* p, double* ap,
                              const double* beta, cudaStream_t st) {
  cr_pupdate_kernel<<<grid_for((long long)g.dim * g.nodes * g.nrhs), 256, 0, st>>>(g, r, ar, p, ap, beta);
  return cudaGetLastError();
}

cudaError_t launch_cg_alpha(int nrhs, const double* pq_part, int nblk, const double* rr, double* alpha, int* active,
                            int* flags, cudaStream_t st) {
  cg_alpha_kernel<<<nrhs, RED_THREADS, 0, st>>>(pq_part, nblk, rr, alpha, active, flags);
  return cudaGetLastError();
}
cudaError_t launch_cg_xr_update(const Geom& g, const double* mw, const double* alpha, const double* p, const double* q,
                                double* x, double* r, double* part, cudaStream_t st) {
  dim3 grd(dot_blocks(g), g.nrhs);
  cg_xr_kernel<<<grd, RED_THREADS, 0, st>>>(g, mw, alpha, p, q, x, r, part);
  return cudaGetLastError();
}
cudaError_t launch_cg_beta(int nrhs, const double* part, int nblk, double* rr, const double* bb, double* beta,
                           double* res, const int* active, cudaStream_t st) {
  cg_beta_kernel<<<nrhs, RED_THREADS, 0, st>>>(part, nblk, rr, bb, beta, res, active);
  return cudaGetLastError();
}

// Device-side control of the CG loop: a while-conditional graph node runs
// one iteration per pass, this kernel last.  It counts the iteration
// (ctl[0]), records its history entry hist[it - 1] (the largest recursive
// relative residual of the active right-hand sides) and ends the loop when
// the host has to act: an FP64 residual replacement is due for an active rhs
// (its residual reached tol = anchor[nrhs], or fell by the factor drop =
// anchor[nrhs + 1] below its anchor), the breakdown flag is set, or the
// window of ctl[1] iterations is used up.
// The host takes the same decisions from the same scalars, so the iterates
// are those of the host-driven loop.
__global__ void cg_control_kernel(cudaGraphConditionalHandle h, int nrhs, const double* __restrict__ res,
                                  const int* __restrict__ active, const double* __restrict__ anchor,
                                  const int* __restrict__ flags, int* __restrict__ ctl, double* __restrict__ hist) {
  const double tol = anchor[nrhs], drop = anchor[nrhs + 1];
  __shared__ double s_max[RED_THREADS];
  __shared__ int s_rep[RED_THREADS];
  double m = 0.0;
  int rep = 0;
  for (int k = threadIdx.x; k < nrhs; k += blockDim.x)
    if (active[k]) {
      const double r = res[k];
      m = fmax(m, r);
      rep |= (r <= tol || (drop > 0.0 && r <= drop * anchor[k])) ? 1 : 0;
    }
  s_max[threadIdx.x] = m;
  s_rep[threadIdx.x] = rep;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s_max[threadIdx.x] = fmax(s_max[threadIdx.x], s_max[threadIdx.x + w]);
      s_rep[threadIdx.x] |= s_rep[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int it = ctl[0] + 1;
    ctl[0] = it;
    hist[it - 1] = s_max[0];
    const bool stop = s_rep[0] != 0 || (*flags & 1) != 0 || it >= ctl[1];
    cudaGraphSetConditional(h, stop ? 0u : 1u);
  }
}
cudaError_t launch_cg_control(cudaGraphConditionalHandle h, int nrhs, const double* res, const int* active,
                              const double* anchor, const int* flags, int* ctl, double* hist, cudaStream_t st) {
  cg_control_kernel<<<1, RED_THREADS, 0, st>>>(h, nrhs, res, active, anchor, flags, ctl, hist);
  return cudaGetLastError();
}

__global__ void axpby_kernel(long long n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}
cudaError_t launch_axpby(long long n, double a, const double* x, double b, double* y, cudaStream_t st) {
  axpby_kernel<<<grid_for(n), 256, 0, st>>>(n, a, x, b, y);
  return cudaGetLastError();
}

// ---- mass weights: rho * (trapezoid or SBP norm product) * h^dim per unknown node
__device__ __forceinline__ double axis_weight(int p, int N, int lo_free, int hi_free, int order) {
  if (order == 4) {
    const int q = p < N - 1 - p ? p : N - 1 - p;
    switch (q) {
      case 0: return 17.0 / 48.0;
      case 1: return 59.0 / 48.0;
      case 2: return 43.0 / 48.0;
      case 3: return 49.0 / 48.0;
      default: return 1.0;
    }
  }
  if ((p == 0 && lo_free) || (p == N - 1 && hi_free)) return 0.5;
  return 1.0;
}

__global__ void fill_mass_kernel(Geom g, int order, const double* __restrict__ rho_full, double hd,
                                 double* __restrict__ mw) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.nodes;
       i += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    node_coords(g, i, x, y, z);
    double w = axis_weight(x, g.n[0], g.lo_free[0], g.hi_free[0], order) *
               axis_weight(y, g.n[1], g.lo_free[1], g.hi_free[1], order);
    if (g.dim == 3) w *= axis_weight(z, g.n[2], g.lo_free[2], g.hi_free[2], order);
    const long long full = ((long long)z * g.n[1] + y) * g.n[0] + x;
    mw[i] = rho_full[full] * w * hd;
  }
}
cudaError_t launch_fill_mass(const Geom& g, int order, const double* rho_full, double h, double* mw,
                             cudaStream_t st) {
  double hd = h * h;
  if (g.dim == 3) hd *= h;
  fill_mass_kernel<<<grid_for(g.nodes), 256, 0, st>>>(g, order, rho_full, hd, mw);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Weighted inner products without any allocation (ewh_mdot_noalloc).
//
// A deterministic two-pass reduction like the context's M inner product (its
// own block count, at most NOALLOC_BLOCKS, so for large vectors the rounding
// differs from ewh_mdot's), with the per-block partial sums in a file-scope
// device array instead of context-owned memory, so the call allocates nothing.  Capacity:
// NOALLOC_BLOCKS blocks per batch member, at most NOALLOC_MAX_BATCH members.
// ---------------------------------------------------------------------------
constexpr int NOALLOC_BLOCKS = 64;
constexpr int NOALLOC_MAX_BATCH = 128;
static __device__ __align__(256) double g_noalloc_partials[NOALLOC_BLOCKS * NOALLOC_MAX_BATCH];

__global__ void noalloc_partial_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                       const double* __restrict__ w, long long nodes, int ncomp,
                                       double* __restrict__ part) {
  const int b = blockIdx.y;
  const long long n = (long long)ncomp * nodes;
  const double* xb = x + (long long)b * n;
  const double* yb = y + (long long)b * n;
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)RED_THREADS + threadIdx.x; i < n;
       i += (long long)gridDim.x * RED_THREADS)
    s += w[i % nodes] * xb[i] * yb[i];
  s = block_sum(s);
  if (threadIdx.x == 0) part[(long long)b * NOALLOC_BLOCKS + blockIdx.x] = s;
}

__global__ void noalloc_final_kernel(const double* __restrict__ part, int nblk, double* __restrict__ out) {
  const int b = blockIdx.x;
  const double s = sum_partials(part + (long long)b * NOALLOC_BLOCKS, nblk);
  if (threadIdx.x == 0) out[b] = s;
}

}  // namespace ewh

#include <mutex>

#include "../../include/ewh.h"

namespace {
// Device address of g_noalloc_partials, fetched once per device with that
// device current (in host code the symbol itself is only a host stand-in).
// The address belongs to the device's current (primary) context: after a
// cudaDeviceReset the module may load at another address, so the cached
// value is tagged with the context it was taken in and looked up again when
// the current context differs.
constexpr int MAX_DEVICES = 64;
double* g_noalloc_ptr[MAX_DEVICES] = {nullptr};
void* g_noalloc_ctx[MAX_DEVICES] = {nullptr};
std::mutex g_noalloc_mutex;

// The calling thread's current CUDA context (driver handle), or null when
// the driver entry point is unavailable.
void* current_cuda_context() {
  typedef int (*GetCurrentFn)(void**);
  static GetCurrentFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<GetCurrentFn>(p);
    else
      cudaGetLastError();
  });
  void* c = nullptr;
  if (fn && fn(&c) != 0) c = nullptr;
  return c;
}
}  // namespace

extern "C" ewh_status ewh_mdot_noalloc(const double* x, const double* y, const double* w, long long nodes,
                                       int ncomp, int nbatch, double* out, void* cuda_stream) {
  using namespace ewh;
  if (!x || !y || !w || !out) {
    set_global_error("ewh_mdot_noalloc: null pointer argument");
    return EWH_EINVAL;
  }
  if (nodes < 1 || ncomp < 1 || nbatch < 1) {
    set_global_error("ewh_mdot_noalloc: nodes, ncomp and nbatch must be >= 1");
    return EWH_EINVAL;
  }
  if (nbatch > NOALLOC_MAX_BATCH) {
    set_global_error("ewh_mdot_noalloc: nbatch exceeds the fixed scratch capacity of 128 batch members");
    return EWH_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
    cudaGetLastError();
    set_global_error("ewh_mdot_noalloc: no usable current CUDA device");
    return EWH_ECUDA;
  }
  double* part = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    void* cur = current_cuda_context();
    if (!g_noalloc_ptr[dev] || (cur && cur != g_noalloc_ctx[dev])) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        set_global_error(std::string("ewh_mdot_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
        return EWH_ECUDA;
      }
      g_noalloc_ptr[dev] = static_cast<double*>(p);
      g_noalloc_ctx[dev] = current_cuda_context();
    }
    part = g_noalloc_ptr[dev];
  }
  const long long n = (long long)ncomp * nodes;
  long long nb = (n + 4 * RED_THREADS - 1) / (4 * RED_THREADS);
  if (nb > NOALLOC_BLOCKS) nb = NOALLOC_BLOCKS;
  if (nb < 1) nb = 1;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // every partial slot read by the final pass is written by the first one, so
  // nothing left over from an earlier call needs clearing
  noalloc_partial_kernel<<<dim3((unsigned)nb, (unsigned)nbatch), RED_THREADS, 0, st>>>(x, y, w, nodes, ncomp, part);
  noalloc_final_kernel<<<nbatch, RED_THREADS, 0, st>>>(part, (int)nb, out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_global_error(std::string("ewh_mdot_noalloc: launch failed: ") + cudaGetErrorString(e));
    return EWH_ECUDA;
  }
  return EWH_OK;
}

namespace ewh {

template cudaError_t launch_pack<float>(const Geom&, const double*, float*, cudaStream_t);
template cudaError_t launch_pack<double>(const Geom&, const double*, double*, cudaStream_t);
template cudaError_t launch_unpack<float>(const Geom&, const float*, double*, const double*, cudaStream_t);
template cudaError_t launch_unpack<double>(const Geom&, const double*, double*, const double*, cudaStream_t);
template cudaError_t launch_pupdate_pack<float>(const Geom&, const double*, double*, const double*, float*,
                                                cudaStream_t);
template cudaError_t launch_pupdate_pack<double>(const Geom&, const double*, double*, const double*, double*,
                                                 cudaStream_t);

}  // namespace ewh
