// C ABI of the El-WaveHoltz library: problem setup (Sections 2.1, 4.1, 4.3),
// WaveHoltz applies (Section 3, eq. qoper) and the Krylov solve of
// M (I - S) v = M Pi 0 (Section 4.5, eq. amat_sym).
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ewh.h"
#include "ewh_internal.cuh"

using namespace ewh;

namespace {

thread_local std::string g_create_error = "no error";

template <typename T>
struct Wave {
  T* u_a = nullptr;
  T* u_b = nullptr;
  T* delta = nullptr;
  T* acc = nullptr;
  T* lam = nullptr;
  T* mu = nullptr;
  T* irh2 = nullptr;
  T* frho = nullptr;   // null when the problem has no forcing
  T* sigma = nullptr;  // order 4 only
  cudaGraphExec_t graph_S = nullptr;
  cudaGraphExec_t graph_Pi0 = nullptr;
  long long graph_S_kernels = 0;
  long long graph_Pi0_kernels = 0;
  bool ready = false;
};

}  // namespace

struct ewh_ctx {
  Geom g{};
  int order = 2;
  int precision = EWH_FP64;
  int periods = 1;
  int corrected = 1;
  int nt = 0;
  double h = 0, omega = 0, omega_t = 0, dt = 0, kt = 0, c = 1;
  std::vector<double> weights;  // periods*nt + 1
  bool has_forcing = false;
  cudaStream_t user_stream = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  Wave<double> w64;
  Wave<float> w32;
  // Krylov state (FP64): x, r, p, q, b, d (correction), tmp
  double *kx = nullptr, *kr = nullptr, *kp = nullptr, *kq = nullptr, *kb = nullptr, *kd = nullptr,
         *ktmp = nullptr;
  double* mw = nullptr;     // mass weight per unknown node
  double* part = nullptr;   // reduction partials [nrhs][nblk]
  double* scal = nullptr;   // per rhs: rr, alpha, beta, bb, res, dot  (6 * nrhs)
  int* active = nullptr;    // per rhs
  int* flags = nullptr;
  double* h_scal = nullptr; // pinned host mirror of scal
  int nblk = 1;
  long long launches = 0;
  std::string err = "no error";
  std::vector<double> history;
  // device timing of wave solves: pending event pairs, reusable events
  struct Timed {
    cudaEvent_t e0, e1;
    int prec;
    long long steps;
  };
  std::vector<Timed> pending;
  std::vector<cudaEvent_t> spare_events;
  double wave_ms[2] = {0, 0};
  long long wave_steps[2] = {0, 0};
  long long wave_count[2] = {0, 0};
};

namespace {

#define EWH_CU(call)                                                                   \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      return fail(ctx, EWH_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    }                                                                                  \
  } while (0)

}  // namespace

void ewh::set_global_error(const std::string& msg) { g_create_error = msg; }

namespace {

ewh_status fail(ewh_ctx* ctx, ewh_status s, const std::string& msg) {
  if (ctx) ctx->err = msg;
  else g_create_error = msg;
  return s;
}

long long total_unknowns(const ewh_ctx* c) { return (long long)c->g.nrhs * c->g.dim * c->g.nodes; }

template <typename T>
cudaError_t alloc_zero(T** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemset(*p, 0, count * sizeof(T));
}

// full-grid FP64 -> padded T (one component), optionally scaled by 1/rho
template <typename T>
__global__ void to_padded_kernel(Geom g, const double* __restrict__ src, const double* __restrict__ rho,
                                 int mode, double h2, T* __restrict__ dst) {
  const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.n[0]);
    const int y = (int)((i / g.n[0]) % g.n[1]);
    const int z = (int)(i / ((long long)g.n[0] * g.n[1]));
    double v;
    if (mode == 0) v = src[i];                       // copy
    else if (mode == 1) v = 1.0 / (rho[i] * h2);     // 1 / (rho h^2)
    else v = is_unknown(g, x, y, z) ? src[i] / rho[i] : 0.0;  // f / rho at unknowns
    dst[pidx(g, 0, 0, x, y, z)] = (T)v;
  }
}

template <typename T>
ewh_status build_wave(ewh_ctx* ctx, Wave<T>& w, const double* d_rho, const double* d_lam, const double* d_mu,
                      const double* d_f) {
  const Geom& g = ctx->g;
  const size_t field = (size_t)g.field;
  const size_t state = field * g.dim * g.nrhs;
  EWH_CU(alloc_zero(&w.u_a, state));
  EWH_CU(alloc_zero(&w.u_b, state));
  EWH_CU(alloc_zero(&w.delta, state));
  EWH_CU(alloc_zero(&w.acc, state));
  EWH_CU(alloc_zero(&w.lam, field));
  EWH_CU(alloc_zero(&w.mu, field));
  EWH_CU(alloc_zero(&w.irh2, field));
  if (ctx->order == 4) EWH_CU(alloc_zero(&w.sigma, field * (g.dim == 2 ? 3 : 6) * g.nrhs));
  const long long full = (long long)g.n[0] * g.n[1] * g.n[2];
  const int blocks = (int)std::min<long long>((full + 255) / 256, 4096);
  const double h2 = ctx->h * ctx->h;
  to_padded_kernel<T><<<blocks, 256, 0, ctx->st>>>(g, d_lam, d_rho, 0, h2, w.lam);
  to_padded_kernel<T><<<blocks, 256, 0, ctx->st>>>(g, d_mu, d_rho, 0, h2, w.mu);
  to_padded_kernel<T><<<blocks, 256, 0, ctx->st>>>(g, d_rho, d_rho, 1, h2, w.irh2);
  ctx->launches += 3;
  if (d_f) {
    EWH_CU(alloc_zero(&w.frho, state));
    for (int r = 0; r < g.nrhs; ++r)
      for (int c = 0; c < g.dim; ++c) {
        to_padded_kernel<T><<<blocks, 256, 0, ctx->st>>>(g, d_f + (size_t)(r * g.dim + c) * full, d_rho, 2, h2,
                                                         w.frho + (size_t)(r * g.dim + c) * field);
        ctx->launches += 1;
      }
  }
  EWH_CU(cudaGetLastError());
  return EWH_OK;
}

template <typename T>
void free_wave(Wave<T>& w) {
  if (w.graph_S) cudaGraphExecDestroy(w.graph_S);
  if (w.graph_Pi0) cudaGraphExecDestroy(w.graph_Pi0);
  cudaFree(w.u_a);
  cudaFree(w.u_b);
  cudaFree(w.delta);
  cudaFree(w.acc);
  cudaFree(w.lam);
  cudaFree(w.mu);
  cudaFree(w.irh2);
  cudaFree(w.frho);
  cudaFree(w.sigma);
  w = Wave<T>();
}

template <typename T>
Wave<T>& wave_of(ewh_ctx* c);
template <>
Wave<double>& wave_of<double>(ewh_ctx* c) { return c->w64; }
template <>
Wave<float>& wave_of<float>(ewh_ctx* c) { return c->w32; }

// Enqueue the nt*periods steps of one wave solve (u^0 already in u_a).
template <typename T>
cudaError_t enqueue_steps(ewh_ctx* ctx, Wave<T>& w, bool forced, long long* nl) {
  const int N = ctx->nt * ctx->periods;
  WaveFields<T> f{};
  f.lam = w.lam;
  f.mu = w.mu;
  f.irh2 = w.irh2;
  f.frho = forced ? w.frho : nullptr;
  f.sigma = w.sigma;
  f.delta = w.delta;
  f.acc = w.acc;
  const double two_pi = 2.0 * M_PI;
  for (int n = 0; n < N; ++n) {
    f.u_cur = (n % 2 == 0) ? w.u_a : w.u_b;
    f.u_next = (n % 2 == 0) ? w.u_b : w.u_a;
    StepScalars s;
    s.kt = ctx->kt;
    s.cosn = std::cos(two_pi * (double)(n % ctx->nt) / (double)ctx->nt);
    s.w0 = ctx->weights[0];
    s.wnew = ctx->weights[n + 1];
    const StepMode mode = (n == 0) ? STEP_FIRST : (n == N - 1 ? STEP_LAST : STEP_MID);
    cudaError_t e = launch_step<T>(ctx->g, ctx->order, f, mode, s, ctx->st, nl);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
ewh_status ensure_graph(ewh_ctx* ctx, bool forced) {
  Wave<T>& w = wave_of<T>(ctx);
  cudaGraphExec_t& ge = forced ? w.graph_Pi0 : w.graph_S;
  long long& nk = forced ? w.graph_Pi0_kernels : w.graph_S_kernels;
  if (ge) return EWH_OK;
  cudaGraph_t graph = nullptr;
  EWH_CU(cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal));
  long long count = 0;
  cudaError_t e = enqueue_steps<T>(ctx, w, forced, &count);
  cudaError_t e2 = cudaStreamEndCapture(ctx->st, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(ctx, EWH_ECUDA, std::string("graph capture failed: ") +
                                    cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(&ge, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(ctx, EWH_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  nk = count;
  return EWH_OK;
}

cudaEvent_t take_event(ewh_ctx* ctx) {
  if (!ctx->spare_events.empty()) {
    cudaEvent_t e = ctx->spare_events.back();
    ctx->spare_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Accumulate the elapsed times of completed timed wave solves (the stream
// must have been synchronised).
void collect_timing(ewh_ctx* ctx) {
  for (auto& t : ctx->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.e0, t.e1) == cudaSuccess) {
      ctx->wave_ms[t.prec] += ms;
      ctx->wave_steps[t.prec] += t.steps;
      ctx->wave_count[t.prec] += 1;
    } else {
      cudaGetLastError();
    }
    ctx->spare_events.push_back(t.e0);
    ctx->spare_events.push_back(t.e1);
  }
  ctx->pending.clear();
}

// Launch a wave-solve graph bracketed by timing events.
template <typename T>
cudaError_t launch_timed_graph(ewh_ctx* ctx, cudaGraphExec_t ge) {
  cudaEvent_t e0 = take_event(ctx), e1 = take_event(ctx);
  if (e0) cudaEventRecord(e0, ctx->st);
  cudaError_t e = cudaGraphLaunch(ge, ctx->st);
  if (e1) cudaEventRecord(e1, ctx->st);
  if (e0 && e1) {
    ewh_ctx::Timed t{e0, e1, sizeof(T) == 8 ? 0 : 1, (long long)ctx->nt * ctx->periods};
    ctx->pending.push_back(t);
    if (ctx->pending.size() > 4096) {  // bound the pool on very long solves
      cudaStreamSynchronize(ctx->st);
      collect_timing(ctx);
    }
  } else {
    if (e0) ctx->spare_events.push_back(e0);
    if (e1) ctx->spare_events.push_back(e1);
  }
  return e;
}

// acc <- wave solve from u^0 = dense v_in (or from rest when v_in is null)
template <typename T>
ewh_status run_wave(ewh_ctx* ctx, const double* v_in, bool forced) {
  Wave<T>& w = wave_of<T>(ctx);
  if (forced && !w.frho) return fail(ctx, EWH_EINVAL, "problem was created without forcing");
  ewh_status s = ensure_graph<T>(ctx, forced);
  if (s != EWH_OK) return s;
  const Geom& g = ctx->g;
  if (v_in) {
    EWH_CU(launch_pack<T>(g, v_in, w.u_a, ctx->st));
    ctx->launches += 1;
  } else {
    EWH_CU(cudaMemsetAsync(w.u_a, 0, sizeof(T) * (size_t)g.field * g.dim * g.nrhs, ctx->st));
  }
  EWH_CU(launch_timed_graph<T>(ctx, forced ? w.graph_Pi0 : w.graph_S));
  ctx->launches += forced ? w.graph_Pi0_kernels : w.graph_S_kernels;
  return EWH_OK;
}

template <typename T>
ewh_status apply_S_T(ewh_ctx* ctx, const double* v_in, double* v_out, const double* sub_from) {
  ewh_status s = run_wave<T>(ctx, v_in, false);
  if (s != EWH_OK) return s;
  EWH_CU(launch_unpack<T>(ctx->g, wave_of<T>(ctx).acc, v_out, sub_from, ctx->st));
  ctx->launches += 1;
  return EWH_OK;
}

void enter(ewh_ctx* ctx) {
  cudaEventRecord(ctx->ev_in, ctx->user_stream);
  cudaStreamWaitEvent(ctx->st, ctx->ev_in, 0);
}
void leave(ewh_ctx* ctx) {
  cudaEventRecord(ctx->ev_out, ctx->st);
  cudaStreamWaitEvent(ctx->user_stream, ctx->ev_out, 0);
}

ewh_status check_async(ewh_ctx* ctx) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, EWH_ECUDA, std::string("pending CUDA error: ") + cudaGetErrorString(e));
  return EWH_OK;
}

// scal layout per rhs block: [0] rr, [1] alpha, [2] beta, [3] bb, [4] res, [5] dot
enum { S_RR = 0, S_ALPHA = 1, S_BETA = 2, S_BB = 3, S_RES = 4, S_DOT = 5, S_N = 6 };

double* sc(ewh_ctx* c, int which) { return c->scal + (size_t)which * c->g.nrhs; }

ewh_status mdot_dev(ewh_ctx* ctx, const double* x, const double* y, double* out_dev) {
  EWH_CU(launch_mdot_partial(ctx->g, ctx->mw, x, y, ctx->part, ctx->st));
  EWH_CU(launch_mdot_final(ctx->g, ctx->part, out_dev, ctx->st));
  ctx->launches += 2;
  return EWH_OK;
}

// r = b - (x - S64 x) in FP64, returns per-rhs relative residual (max) on host
ewh_status true_residual(ewh_ctx* ctx, const double* x, double* r, double* max_rel) {
  const Geom& g = ctx->g;
  const int R = g.nrhs;
  const long long n = total_unknowns(ctx);
  // ktmp = x - S x  ; r = b - ktmp
  ewh_status s = apply_S_T<double>(ctx, x, ctx->ktmp, x);
  if (s != EWH_OK) return s;
  EWH_CU(cudaMemcpyAsync(r, ctx->kb, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->st));
  EWH_CU(launch_axpby(n, -1.0, ctx->ktmp, 1.0, r, ctx->st));
  ctx->launches += 1;
  s = mdot_dev(ctx, r, r, sc(ctx, S_DOT));
  if (s != EWH_OK) return s;
  EWH_CU(cudaMemcpyAsync(ctx->h_scal, ctx->scal, sizeof(double) * S_N * R, cudaMemcpyDeviceToHost, ctx->st));
  EWH_CU(cudaStreamSynchronize(ctx->st));
  double worst = 0.0;
  for (int k = 0; k < R; ++k)
    worst = std::max(worst, std::sqrt(ctx->h_scal[S_DOT * R + k] / ctx->h_scal[S_BB * R + k]));
  *max_rel = worst;
  return EWH_OK;
}

// CG in the M inner product on (I - S_T) x = b, S_T the wave solve in
// precision T.  On entry x holds the iterate and r its true FP64 residual.
// Residual replacement (van der Vorst and Ye, "Residual replacement strategies
// for Krylov subspace iterative methods", 2000): whenever the recursive
// residual of an active rhs has dropped by the factor `drop` since the last
// replacement, or reaches tol, r is replaced by the true residual b - A64 x
// (FP64 S apply) while the search direction is kept.  Convergence is declared
// on the true residual only.  drop = 0 replaces only at convergence.
template <typename T>
ewh_status run_cg(ewh_ctx* ctx, double* x, double* r, double tol, int maxit, double drop, ewh_solve_info* inf,
                  double* rel_out) {
  const Geom& g = ctx->g;
  const int R = g.nrhs;
  const long long n = total_unknowns(ctx);
  Wave<T>& w = wave_of<T>(ctx);
  ewh_status st = ensure_graph<T>(ctx, false);
  if (st != EWH_OK) return st;
  // rr = (r, r)_M ; p = 0 ; beta = 0
  st = mdot_dev(ctx, r, r, sc(ctx, S_RR));
  if (st != EWH_OK) return st;
  EWH_CU(cudaMemsetAsync(ctx->kp, 0, sizeof(double) * n, ctx->st));
  EWH_CU(cudaMemsetAsync(sc(ctx, S_BETA), 0, sizeof(double) * R, ctx->st));
  EWH_CU(cudaMemsetAsync(ctx->flags, 0, sizeof(int), ctx->st));
  EWH_CU(cudaMemcpyAsync(ctx->h_scal, ctx->scal, sizeof(double) * S_N * R, cudaMemcpyDeviceToHost, ctx->st));
  EWH_CU(cudaStreamSynchronize(ctx->st));
  std::vector<int> act(R, 1);
  std::vector<double> anchor(R), true_res(R);
  for (int k = 0; k < R; ++k) {
    true_res[k] = std::sqrt(ctx->h_scal[S_RR * R + k] / ctx->h_scal[S_BB * R + k]);
    anchor[k] = true_res[k];
    if (true_res[k] <= tol) act[k] = 0;
  }
  EWH_CU(cudaMemcpyAsync(ctx->active, act.data(), sizeof(int) * R, cudaMemcpyHostToDevice, ctx->st));
  auto worst_true = [&]() {
    double m = 0.0;
    for (int k = 0; k < R; ++k) m = std::max(m, true_res[k]);
    return m;
  };
  ctx->history.push_back(worst_true());
  bool any = false;
  for (int k = 0; k < R; ++k) any = any || act[k];
  int it = 0;
  while (any && inf->iters < maxit) {
    // p = r + beta p ; u^0 = p
    EWH_CU(launch_pupdate_pack<T>(g, r, ctx->kp, sc(ctx, S_BETA), w.u_a, ctx->st));
    ctx->launches += 1;
    EWH_CU(launch_timed_graph<T>(ctx, w.graph_S));
    ctx->launches += w.graph_S_kernels;
    // q = p - S p
    EWH_CU(launch_unpack<T>(g, w.acc, ctx->kq, ctx->kp, ctx->st));
    EWH_CU(launch_mdot_partial(g, ctx->mw, ctx->kp, ctx->kq, ctx->part, ctx->st));
    EWH_CU(launch_cg_alpha(R, ctx->part, ctx->nblk, sc(ctx, S_RR), sc(ctx, S_ALPHA), ctx->active, ctx->flags,
                           ctx->st));
    EWH_CU(launch_cg_xr_update(g, ctx->mw, sc(ctx, S_ALPHA), ctx->kp, ctx->kq, x, r, ctx->part, ctx->st));
    EWH_CU(launch_cg_beta(R, ctx->part, ctx->nblk, sc(ctx, S_RR), sc(ctx, S_BB), sc(ctx, S_BETA),
                          sc(ctx, S_RES), ctx->active, ctx->st));
    ctx->launches += 5;
    ++it;
    ++inf->iters;
    if (sizeof(T) == 8) ++inf->s_applies_fp64;
    else ++inf->s_applies;
    int flag = 0;
    EWH_CU(cudaMemcpyAsync(ctx->h_scal, ctx->scal, sizeof(double) * S_N * R, cudaMemcpyDeviceToHost, ctx->st));
    EWH_CU(cudaMemcpyAsync(act.data(), ctx->active, sizeof(int) * R, cudaMemcpyDeviceToHost, ctx->st));
    EWH_CU(cudaMemcpyAsync(&flag, ctx->flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    EWH_CU(cudaStreamSynchronize(ctx->st));
    if (flag & 1) {
      *rel_out = worst_true();
      return fail(ctx, EWH_EBREAKDOWN, "CG breakdown: (p, (I-S)p)_M <= 0 (indefinite system near resonance)");
    }
    bool replace = false;
    double hist = 0.0;
    for (int k = 0; k < R; ++k) {
      const double res = ctx->h_scal[S_RES * R + k];
      if (act[k]) {
        hist = std::max(hist, res);
        if (res <= tol || (drop > 0.0 && res <= drop * anchor[k])) replace = true;
      }
    }
    ctx->history.push_back(hist);
    if (replace) {
      double dummy = 0.0;
      st = true_residual(ctx, x, r, &dummy);
      if (st != EWH_OK) return st;
      ++inf->s_applies_fp64;
      EWH_CU(launch_cg_replace(R, sc(ctx, S_DOT), sc(ctx, S_RR), sc(ctx, S_BETA), sc(ctx, S_RES), sc(ctx, S_BB),
                               ctx->st));
      ctx->launches += 1;
      bool changed = false;
      for (int k = 0; k < R; ++k) {
        true_res[k] = std::sqrt(ctx->h_scal[S_DOT * R + k] / ctx->h_scal[S_BB * R + k]);
        anchor[k] = true_res[k];
        if (act[k] && true_res[k] <= tol) {
          act[k] = 0;
          changed = true;
        }
      }
      if (changed) EWH_CU(cudaMemcpyAsync(ctx->active, act.data(), sizeof(int) * R, cudaMemcpyHostToDevice, ctx->st));
    }
    any = false;
    for (int k = 0; k < R; ++k) any = any || act[k];
  }
  *rel_out = worst_true();
  (void)it;
  return EWH_OK;
}

ewh_status solve_impl(ewh_ctx* ctx, double tol, int maxit, const double* x0, double* v_out,
                      ewh_solve_info* inf) {
  const Geom& g = ctx->g;
  const long long n = total_unknowns(ctx);
  ctx->history.clear();
  // b = Pi 0 in FP64: the right-hand side every residual is measured against
  ewh_status s = run_wave<double>(ctx, nullptr, true);
  if (s != EWH_OK) return s;
  EWH_CU(launch_unpack<double>(g, ctx->w64.acc, ctx->kb, nullptr, ctx->st));
  ctx->launches += 1;
  inf->s_applies_fp64 += 1;
  s = mdot_dev(ctx, ctx->kb, ctx->kb, sc(ctx, S_BB));
  if (s != EWH_OK) return s;
  double rel = 1.0;
  if (x0) {
    EWH_CU(cudaMemcpyAsync(ctx->kx, x0, sizeof(double) * n, cudaMemcpyDefault, ctx->st));
    s = true_residual(ctx, ctx->kx, ctx->kr, &rel);
    if (s != EWH_OK) return s;
    inf->s_applies_fp64 += 1;
  } else {
    EWH_CU(cudaMemsetAsync(ctx->kx, 0, sizeof(double) * n, ctx->st));
    EWH_CU(cudaMemcpyAsync(ctx->kr, ctx->kb, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->st));
  }
  // FP64: replacement only to confirm convergence.  FP32 stencil: replace
  // every time the recursive residual fell tenfold, so the FP32 operator's
  // rounding never accumulates in the residual beyond one decade.
  ewh_status result;
  if (ctx->precision == EWH_FP64) {
    result = run_cg<double>(ctx, ctx->kx, ctx->kr, tol, maxit, 0.0, inf, &rel);
  } else {
    result = run_cg<float>(ctx, ctx->kx, ctx->kr, tol, maxit, 0.1, inf, &rel);
    if (result == EWH_EBREAKDOWN) {
      // The FP32 operator lost definiteness on the modes nearest resonance
      // (its rounding exceeds their eigenvalues of I - S): continue with the
      // FP64 operator from the current iterate and its true residual.
      s = true_residual(ctx, ctx->kx, ctx->kr, &rel);
      if (s != EWH_OK) return s;
      ++inf->s_applies_fp64;
      ctx->err = "no error";
      result = run_cg<double>(ctx, ctx->kx, ctx->kr, tol, maxit, 0.0, inf, &rel);
    }
  }
  if (result != EWH_OK && result != EWH_EBREAKDOWN) return result;
  inf->rel_res = rel;
  EWH_CU(cudaMemcpyAsync(v_out, ctx->kx, sizeof(double) * n, cudaMemcpyDefault, ctx->st));
  EWH_CU(cudaStreamSynchronize(ctx->st));
  if (result == EWH_EBREAKDOWN) return result;
  if (!(rel <= tol)) {
    return fail(ctx, EWH_ENOTCONV, "not converged: relative residual " + std::to_string(rel) + " > tol after " +
                                       std::to_string(inf->iters) + " iterations");
  }
  return EWH_OK;
}

ewh_status validate_desc(const ewh_grid_desc* d, int nrhs) {
  if (!d) return fail(nullptr, EWH_EINVAL, "desc is NULL");
  if (d->dim != 2 && d->dim != 3) return fail(nullptr, EWH_EINVAL, "dim must be 2 or 3");
  if (d->order != 2 && d->order != 4) return fail(nullptr, EWH_EINVAL, "order must be 2 or 4");
  const int minn = d->order == 4 ? 8 : 4;
  for (int a = 0; a < d->dim; ++a)
    if (d->n[a] < minn || d->n[a] > (1 << 20))
      return fail(nullptr, EWH_EINVAL, "n[" + std::to_string(a) + "] must be in [" + std::to_string(minn) + ", 2^20]");
  for (int k = 0; k < 2 * d->dim; ++k)
    if (d->bc[k] != EWH_BC_DIRICHLET && d->bc[k] != EWH_BC_FREE)
      return fail(nullptr, EWH_EINVAL, "bc entries must be EWH_BC_DIRICHLET or EWH_BC_FREE");
  if (!(d->h > 0.0) || !std::isfinite(d->h)) return fail(nullptr, EWH_EINVAL, "h must be positive and finite");
  if (d->precision != EWH_FP64 && d->precision != EWH_FP32_STENCIL)
    return fail(nullptr, EWH_EINVAL, "precision must be EWH_FP64 or EWH_FP32_STENCIL");
  const double cfl = d->cfl == 0.0 ? 0.5 : d->cfl;
  if (!(cfl > 0.0 && cfl < 1.0)) return fail(nullptr, EWH_EINVAL, "cfl must lie in (0, 1)");
  if (d->periods < 1 || d->periods > 1000) return fail(nullptr, EWH_EINVAL, "periods must be in [1, 1000]");
  if (d->nt < 0 || (d->nt > 0 && d->nt < 5)) return fail(nullptr, EWH_EINVAL, "nt must be 0 or >= 5");
  if (nrhs < 1 || nrhs > 65535) return fail(nullptr, EWH_EINVAL, "nrhs must be in [1, 65535]");
  return EWH_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* ewh_status_string(int s) {
  switch (s) {
    case EWH_OK: return "EWH_OK";
    case EWH_EINVAL: return "EWH_EINVAL";
    case EWH_ENOMEM: return "EWH_ENOMEM";
    case EWH_ECUDA: return "EWH_ECUDA";
    case EWH_ENOTCONV: return "EWH_ENOTCONV";
    case EWH_EBREAKDOWN: return "EWH_EBREAKDOWN";
    case EWH_ETIMEOUT: return "EWH_ETIMEOUT";
    default: return "EWH_UNKNOWN";
  }
}

const char* ewh_last_error(const ewh_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

void ewh_destroy(ewh_ctx* ctx) {
  if (!ctx) return;
  if (ctx->st) cudaStreamSynchronize(ctx->st);
  free_wave(ctx->w64);
  free_wave(ctx->w32);
  cudaFree(ctx->kx);
  cudaFree(ctx->kr);
  cudaFree(ctx->kp);
  cudaFree(ctx->kq);
  cudaFree(ctx->kb);
  cudaFree(ctx->kd);
  cudaFree(ctx->ktmp);
  cudaFree(ctx->mw);
  cudaFree(ctx->part);
  cudaFree(ctx->scal);
  cudaFree(ctx->active);
  cudaFree(ctx->flags);
  if (ctx->h_scal) cudaFreeHost(ctx->h_scal);
  for (auto& t : ctx->pending) {
    cudaEventDestroy(t.e0);
    cudaEventDestroy(t.e1);
  }
  for (auto e : ctx->spare_events) cudaEventDestroy(e);
  if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
  if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
  if (ctx->st) cudaStreamDestroy(ctx->st);
  delete ctx;
}

ewh_status ewh_create(const ewh_grid_desc* desc, const double* rho, const double* lambda, const double* mu,
                      double omega, const double* forcing, int nrhs, void* cuda_stream, ewh_ctx** out) {
  if (!out) return fail(nullptr, EWH_EINVAL, "out is NULL");
  *out = nullptr;
  ewh_status vs = validate_desc(desc, nrhs);
  if (vs != EWH_OK) return vs;
  if (!rho || !lambda || !mu) return fail(nullptr, EWH_EINVAL, "rho, lambda and mu are required");
  if (!(omega > 0.0) || !std::isfinite(omega)) return fail(nullptr, EWH_EINVAL, "omega must be positive and finite");
  const int dim = desc->dim;
  const long long full = (long long)desc->n[0] * desc->n[1] * (dim == 3 ? desc->n[2] : 1);
  // media on the host for validation and the time-step bound
  std::vector<double> hr(full), hl(full), hm(full);
  auto fetch = [&](const double* src, std::vector<double>& dst) -> cudaError_t {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, src) == cudaSuccess &&
        (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged))
      return cudaMemcpy(dst.data(), src, sizeof(double) * full, cudaMemcpyDeviceToHost);
    cudaGetLastError();  // host memory (or no device): plain copy
    std::memcpy(dst.data(), src, sizeof(double) * full);
    return cudaSuccess;
  };
  if (fetch(rho, hr) != cudaSuccess || fetch(lambda, hl) != cudaSuccess || fetch(mu, hm) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, EWH_EINVAL, "cannot read rho/lambda/mu");
  }
  double speed2 = 0.0;
  for (long long i = 0; i < full; ++i) {
    const double r = hr[i], l = hl[i], m = hm[i];
    if (!std::isfinite(r) || !std::isfinite(l) || !std::isfinite(m) || !(r > 0.0) || !(m > 0.0) ||
        !(l > -2.0 * m / dim))
      return fail(nullptr, EWH_EINVAL,
                  "invalid medium at node " + std::to_string(i) + ": need finite rho > 0, mu > 0, lambda > -2 mu / dim");
    const double c2 = (l + (dim + 1) * m) / r;
    if (c2 > speed2) speed2 = c2;
  }

  ewh_ctx* ctx = new ewh_ctx();
  ctx->order = desc->order;
  ctx->precision = desc->precision;
  ctx->periods = desc->periods;
  ctx->corrected = desc->corrected ? 1 : 0;
  ctx->h = desc->h;
  ctx->omega = omega;
  ctx->user_stream = (cudaStream_t)cuda_stream;
  Geom& g = ctx->g;
  g.dim = dim;
  g.nrhs = nrhs;
  for (int a = 0; a < 3; ++a) {
    g.n[a] = a < dim ? desc->n[a] : 1;
    g.lo_free[a] = a < dim ? (desc->bc[2 * a] == EWH_BC_FREE) : 1;
    g.hi_free[a] = a < dim ? (desc->bc[2 * a + 1] == EWH_BC_FREE) : 1;
  }
  for (int a = 0; a < 3; ++a) {
    if (a < dim) {
      const int rounded = ((g.n[a] + TILE_ROUND - 1) / TILE_ROUND) * TILE_ROUND;
      g.np[a] = rounded + 2 * PAD;
      g.off[a] = g.lo_free[a] ? 0 : 1;
      g.nu[a] = g.n[a] - (g.lo_free[a] ? 0 : 1) - (g.hi_free[a] ? 0 : 1);
    } else {
      g.np[a] = 1;
      g.off[a] = 0;
      g.nu[a] = 1;
    }
  }
  g.pz = dim == 3 ? PAD : 0;
  g.plane = (long long)g.np[0] * g.np[1];
  g.field = g.plane * g.np[2];
  g.nodes = (long long)g.nu[0] * g.nu[1] * g.nu[2];

  // time step (Section 4.3): dt_CFL, nt, dt, w~, c, kt and trapezoid weights
  const double cfl = desc->cfl == 0.0 ? 0.5 : desc->cfl;
  const double T = 2.0 * M_PI / omega;
  const double dtc = cfl * desc->h / std::sqrt(speed2);
  int nt = desc->nt;
  if (nt == 0) {
    const double q = std::ceil(T / dtc);
    if (q > 1e7) {
      delete ctx;
      return fail(nullptr, EWH_EINVAL, "more than 1e7 time steps per period");
    }
    nt = std::max(5, (int)q);
  }
  ctx->nt = nt;
  ctx->dt = T / nt;
  ctx->omega_t = 2.0 * std::sin(omega * ctx->dt / 2.0) / ctx->dt;
  ctx->c = ctx->corrected ? (ctx->omega_t / omega) * (ctx->omega_t / omega) : 1.0;
  ctx->kt = ctx->c * ctx->dt * ctx->dt;
  const int N = nt * ctx->periods;
  ctx->weights.resize(N + 1);
  for (int k = 0; k <= N; ++k) {
    const double eta = (k == 0 || k == N) ? 0.5 : 1.0;
    ctx->weights[k] = (2.0 / N) * eta * (std::cos(2.0 * M_PI * k / nt) - 0.25);
  }
  ctx->has_forcing = forcing != nullptr;

  // CUDA resources
  auto bail = [&](ewh_status s, const std::string& m) {
    g_create_error = m;
    ewh_destroy(ctx);
    return s;
  };
  if (cudaStreamCreateWithFlags(&ctx->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return bail(EWH_ECUDA, "cannot create stream/events (no CUDA device?)");
  }
  enter(ctx);
  double *d_r = nullptr, *d_l = nullptr, *d_m = nullptr, *d_f = nullptr;
  const size_t fbytes = sizeof(double) * (size_t)full * dim * nrhs;
  bool ok = cudaMalloc(&d_r, sizeof(double) * full) == cudaSuccess &&
            cudaMalloc(&d_l, sizeof(double) * full) == cudaSuccess &&
            cudaMalloc(&d_m, sizeof(double) * full) == cudaSuccess &&
            (!forcing || cudaMalloc(&d_f, fbytes) == cudaSuccess);
  if (!ok) {
    cudaGetLastError();
    cudaFree(d_r);
    cudaFree(d_l);
    cudaFree(d_m);
    cudaFree(d_f);
    return bail(EWH_ENOMEM, "device allocation of the medium failed");
  }
  cudaMemcpyAsync(d_r, hr.data(), sizeof(double) * full, cudaMemcpyHostToDevice, ctx->st);
  cudaMemcpyAsync(d_l, hl.data(), sizeof(double) * full, cudaMemcpyHostToDevice, ctx->st);
  cudaMemcpyAsync(d_m, hm.data(), sizeof(double) * full, cudaMemcpyHostToDevice, ctx->st);
  if (forcing) cudaMemcpyAsync(d_f, forcing, fbytes, cudaMemcpyDefault, ctx->st);

  ewh_status s = build_wave<double>(ctx, ctx->w64, d_r, d_l, d_m, d_f);
  if (s == EWH_OK && ctx->precision == EWH_FP32_STENCIL) s = build_wave<float>(ctx, ctx->w32, d_r, d_l, d_m, d_f);
  const long long n = total_unknowns(ctx);
  ctx->nblk = dot_blocks(g);
  if (s == EWH_OK) {
    ok = alloc_zero(&ctx->kx, n) == cudaSuccess && alloc_zero(&ctx->kr, n) == cudaSuccess &&
         alloc_zero(&ctx->kp, n) == cudaSuccess && alloc_zero(&ctx->kq, n) == cudaSuccess &&
         alloc_zero(&ctx->kb, n) == cudaSuccess && alloc_zero(&ctx->kd, n) == cudaSuccess &&
         alloc_zero(&ctx->ktmp, n) == cudaSuccess && alloc_zero(&ctx->mw, g.nodes) == cudaSuccess &&
         alloc_zero(&ctx->part, (size_t)ctx->nblk * nrhs) == cudaSuccess &&
         alloc_zero(&ctx->scal, (size_t)S_N * nrhs) == cudaSuccess &&
         alloc_zero(&ctx->active, nrhs) == cudaSuccess && alloc_zero(&ctx->flags, 1) == cudaSuccess &&
         cudaMallocHost(&ctx->h_scal, sizeof(double) * S_N * nrhs) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      s = fail(ctx, EWH_ENOMEM, "device allocation of the Krylov workspace failed");
    }
  }
  if (s == EWH_OK) {
    if (launch_fill_mass(g, ctx->order, d_r, desc->h, ctx->mw, ctx->st) != cudaSuccess)
      s = fail(ctx, EWH_ECUDA, "mass kernel launch failed");
    ctx->launches += 1;
  }
  cudaError_t e = cudaStreamSynchronize(ctx->st);
  cudaFree(d_r);
  cudaFree(d_l);
  cudaFree(d_m);
  cudaFree(d_f);
  if (s == EWH_OK && e != cudaSuccess) s = fail(ctx, EWH_ECUDA, std::string("setup: ") + cudaGetErrorString(e));
  if (s != EWH_OK) {
    std::string m = ctx->err;
    if (m == "no error") m = g_create_error;
    return bail(s, m);
  }
  leave(ctx);
  *out = ctx;
  return EWH_OK;
}

ewh_status ewh_get_info(const ewh_ctx* ctx, ewh_problem_info* info) {
  if (!ctx || !info) return EWH_EINVAL;
  info->nt = ctx->nt;
  info->periods = ctx->periods;
  info->dt = ctx->dt;
  info->omega = ctx->omega;
  info->omega_tilde = ctx->omega_t;
  info->kt = ctx->kt;
  info->nodes = ctx->g.nodes;
  info->n_unknowns = (long long)ctx->g.dim * ctx->g.nodes;
  info->nrhs = ctx->g.nrhs;
  for (int a = 0; a < 3; ++a) info->nu[a] = ctx->g.nu[a];
  return EWH_OK;
}

static ewh_status apply_S_common(ewh_ctx* ctx, const double* v_in, double* v_out, bool force64) {
  if (!ctx || !v_in || !v_out) return fail(ctx, EWH_EINVAL, "null argument");
  ewh_status s = check_async(ctx);
  if (s != EWH_OK) return s;
  enter(ctx);
  if (ctx->precision == EWH_FP64 || force64) s = apply_S_T<double>(ctx, v_in, v_out, nullptr);
  else s = apply_S_T<float>(ctx, v_in, v_out, nullptr);
  leave(ctx);
  if (s == EWH_OK) s = check_async(ctx);
  return s;
}

ewh_status ewh_apply_S(ewh_ctx* ctx, const double* v_in, double* v_out) {
  return apply_S_common(ctx, v_in, v_out, false);
}

ewh_status ewh_apply_S_fp64(ewh_ctx* ctx, const double* v_in, double* v_out) {
  return apply_S_common(ctx, v_in, v_out, true);
}

ewh_status ewh_apply_Pi0(ewh_ctx* ctx, double* b_out) {
  if (!ctx || !b_out) return fail(ctx, EWH_EINVAL, "null argument");
  ewh_status s = check_async(ctx);
  if (s != EWH_OK) return s;
  enter(ctx);
  if (ctx->precision == EWH_FP64) {
    s = run_wave<double>(ctx, nullptr, true);
    if (s == EWH_OK && launch_unpack<double>(ctx->g, ctx->w64.acc, b_out, nullptr, ctx->st) != cudaSuccess)
      s = fail(ctx, EWH_ECUDA, "unpack launch failed");
  } else {
    s = run_wave<float>(ctx, nullptr, true);
    if (s == EWH_OK && launch_unpack<float>(ctx->g, ctx->w32.acc, b_out, nullptr, ctx->st) != cudaSuccess)
      s = fail(ctx, EWH_ECUDA, "unpack launch failed");
  }
  ctx->launches += 1;
  leave(ctx);
  if (s == EWH_OK) s = check_async(ctx);
  return s;
}

ewh_status ewh_apply_minvK(ewh_ctx* ctx, const double* u, double* out) {
  if (!ctx || !u || !out) return fail(ctx, EWH_EINVAL, "null argument");
  ewh_status s = check_async(ctx);
  if (s != EWH_OK) return s;
  enter(ctx);
  Wave<double>& w = ctx->w64;
  if (launch_pack<double>(ctx->g, u, w.u_a, ctx->st) != cudaSuccess ||
      launch_minvK<double>(ctx->g, ctx->order, w.u_a, w.u_b, w.lam, w.mu, w.irh2, w.sigma, ctx->st,
                           &ctx->launches) != cudaSuccess ||
      launch_unpack<double>(ctx->g, w.u_b, out, nullptr, ctx->st) != cudaSuccess)
    s = fail(ctx, EWH_ECUDA, "operator launch failed");
  ctx->launches += 2;
  leave(ctx);
  if (s == EWH_OK) s = check_async(ctx);
  return s;
}

ewh_status ewh_mdot(ewh_ctx* ctx, const double* x, const double* y, double* out) {
  if (!ctx || !x || !y || !out) return fail(ctx, EWH_EINVAL, "null argument");
  ewh_status s = check_async(ctx);
  if (s != EWH_OK) return s;
  enter(ctx);
  s = mdot_dev(ctx, x, y, sc(ctx, S_DOT));
  if (s == EWH_OK) {
    if (cudaMemcpyAsync(out, sc(ctx, S_DOT), sizeof(double) * ctx->g.nrhs, cudaMemcpyDeviceToHost, ctx->st) !=
            cudaSuccess ||
        cudaStreamSynchronize(ctx->st) != cudaSuccess)
      s = fail(ctx, EWH_ECUDA, "mdot copy failed");
  }
  leave(ctx);
  return s;
}

ewh_status ewh_solve(ewh_ctx* ctx, double tol, int maxit, const double* x0_or_null, double* v_out,
                     ewh_solve_info* info) {
  if (!ctx || !v_out) return fail(ctx, EWH_EINVAL, "null argument");
  if (!(tol > 0.0) || maxit < 0) return fail(ctx, EWH_EINVAL, "tol must be > 0 and maxit >= 0");
  if (!ctx->has_forcing) return fail(ctx, EWH_EINVAL, "problem was created without forcing");
  ewh_status s = check_async(ctx);
  if (s != EWH_OK) return s;
  const auto t0 = std::chrono::steady_clock::now();
  enter(ctx);
  ewh_solve_info inf{};
  s = solve_impl(ctx, tol, maxit, x0_or_null, v_out, &inf);
  leave(ctx);
  cudaStreamSynchronize(ctx->st);
  inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  inf.status = s;
  if (info) *info = inf;
  if (s == EWH_OK) s = check_async(ctx);
  return s;
}

ewh_status ewh_residual_history(const ewh_ctx* ctx, double* out, int cap, int* count) {
  if (!ctx || !count) return EWH_EINVAL;
  *count = (int)ctx->history.size();
  if (out)
    for (int i = 0; i < cap && i < *count; ++i) out[i] = ctx->history[i];
  return EWH_OK;
}

long long ewh_kernel_launches(const ewh_ctx* ctx) { return ctx ? ctx->launches : 0; }

ewh_status ewh_get_stats(ewh_ctx* ctx, ewh_stats* out) {
  if (!ctx || !out) return EWH_EINVAL;
  if (cudaStreamSynchronize(ctx->st) != cudaSuccess) return fail(ctx, EWH_ECUDA, "synchronise failed");
  collect_timing(ctx);
  for (int k = 0; k < 2; ++k) {
    out->wave_ms[k] = ctx->wave_ms[k];
    out->steps[k] = ctx->wave_steps[k];
    out->waves[k] = ctx->wave_count[k];
  }
  out->launches = ctx->launches;
  return EWH_OK;
}

ewh_status ewh_reset_stats(ewh_ctx* ctx) {
  if (!ctx) return EWH_EINVAL;
  if (cudaStreamSynchronize(ctx->st) != cudaSuccess) return fail(ctx, EWH_ECUDA, "synchronise failed");
  collect_timing(ctx);
  for (int k = 0; k < 2; ++k) ctx->wave_ms[k] = 0, ctx->wave_steps[k] = 0, ctx->wave_count[k] = 0;
  ctx->launches = 0;
  return EWH_OK;
}

}  // extern "C"
