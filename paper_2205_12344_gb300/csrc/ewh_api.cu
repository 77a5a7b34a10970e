// C ABI of the El-WaveHoltz library: problem setup (Sections 2.1, 4.1, 4.3),
// WaveHoltz applies (Section 3, eq. qoper) and the Krylov solve of
// M (I - S) v = M Pi 0 (Section 4.5, eq. amat_sym).
#include <cuda_runtime.h>

#include <type_traits>

#include <sys/stat.h>
#include <unistd.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cctype>
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
  T* sigma = nullptr;  // order 4 only (mapped grids: the four fluxes)
  T* met = nullptr;    // mapped grids: metric planes (y_r, -x_r, -y_q, x_q); lam, mu hold lambda / J, mu / J
  cudaGraphExec_t graph_S = nullptr;
  cudaGraphExec_t graph_Pi0 = nullptr;
  long long graph_S_kernels = 0;
  long long graph_Pi0_kernels = 0;
  int variant = -1;           // step-kernel variant (autotuner), -1 = not chosen yet
  int fallback = 0;           // fastest variant that is not the resident solve
  float variant_ms[YM_VARIANT + 1] = {};  // per time level
  bool ready = false;
  // on-chip resident solve (2D order 4 FP32, one rhs): per-level scalars,
  // barrier words and the partition per CTA shape
  double* d_cosn = nullptr;
  double* d_wnew = nullptr;
  unsigned* bar = nullptr;
  ResidentPlan rplan[RS_SHAPES];
  // fused marching FP32 order-4 step (3D z-march, 2D y-march): bulk-tensor
  // maps of u_a / u_b, grid (control words in bar)
  ZmPlan zm;
  // CG iterations under device control (a while-conditional graph): 0 not
  // built yet, 1 built, -1 unavailable (the host drives every iteration)
  cudaGraphExec_t cg_loop = nullptr;
  int cg_loop_state = 0;
  long long cg_loop_kernels = 0;  // kernels of one pass
};

// step-kernel variants of the 2D order-4 FP32 solve beyond the launcher's
// own (split tiles 0..3, fused 4): 5 + shape = resident solve of that shape
constexpr int VARIANT_RESIDENT = 5;
// least nodes per CTA block of a batch member's on-chip solve (resident_ok)
constexpr long long RS_BATCH_MIN_BLOCK = 2048;
// longest window of CG iterations under device control between host polls
constexpr int CG_WINDOW_MAX = 256;
static_assert(VARIANT_RESIDENT + RS_SHAPES == YM_VARIANT, "2D order-4 variants: split 0..3, fused 4, resident, y-march");
inline bool is_resident_variant(int v) { return v >= VARIANT_RESIDENT && v < VARIANT_RESIDENT + RS_SHAPES; }

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
  double *kar = nullptr, *kap = nullptr;  // conjugate residual: A r, A p
  double* mw = nullptr;     // mass weight per unknown node
  double* part = nullptr;   // reduction partials [nrhs][nblk]
  double* scal = nullptr;   // per rhs: rr, alpha, beta, bb, res, dot  (6 * nrhs)
  int* active = nullptr;    // per rhs
  int* flags = nullptr;
  double* h_scal = nullptr; // pinned host mirror of scal
  int* h_act = nullptr;     // pinned host mirror of active (nrhs)
  int* h_flag = nullptr;    // pinned host mirror of flags
  // device-side CG loop control: per-rhs replacement anchors then tol and
  // drop (nrhs + 2), [0] iterations of the current window, [1] window length,
  // the window's history; pinned mirrors
  double* d_anchor = nullptr;
  int* d_loop = nullptr;
  double* d_hist = nullptr;
  double* h_anchor = nullptr;
  int* h_loop = nullptr;
  double* h_hist = nullptr;
  int nblk = 1;
  long long launches = 0;
  // implicit scheme (Section 4.4; FP64, dense unknown layout): level vectors,
  // inner-solve vectors, f/rho, device scalars of the inner CG
  bool batch_member = false;  // member of an ewh_batch (see resident_ok)
  int implicit = 0;
  double alpha = 2.0;
  double *iu_prev = nullptr, *iu = nullptr, *iu_next = nullptr, *ig = nullptr, *ir = nullptr, *ip = nullptr,
         *iq = nullptr, *iacc = nullptr, *ifr = nullptr, *iscal = nullptr;
  long long inner_iters = 0;  // inner CG iterations of the implicit levels (accounting)
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
  long long grid_timeouts_base = 0;  // grid-wait give-ups counted before the last ewh_reset_stats
  long long loop_steps[2] = {0, 0};   // levels / wave solves inside device-controlled CG windows
  long long loop_waves[2] = {0, 0};
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
cudaError_t alloc_zero(T** p, size_t count, cudaStream_t st) {
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) return e;
  // zeroed on the context's (non-blocking) stream, ahead of the kernels that fill it
  return cudaMemsetAsync(*p, 0, count * sizeof(T), st);
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
                      const double* d_f, const double* d_met) {
  const Geom& g = ctx->g;
  const size_t field = (size_t)g.field;
  const size_t state = field * g.dim * g.nrhs;
  EWH_CU(alloc_zero(&w.u_a, state, ctx->st));
  EWH_CU(alloc_zero(&w.u_b, state, ctx->st));
  EWH_CU(alloc_zero(&w.delta, state, ctx->st));
  EWH_CU(alloc_zero(&w.acc, state, ctx->st));
  EWH_CU(alloc_zero(&w.lam, field, ctx->st));
  EWH_CU(alloc_zero(&w.mu, field, ctx->st));
  EWH_CU(alloc_zero(&w.irh2, field, ctx->st));
  if (ctx->order == 4) EWH_CU(alloc_zero(&w.sigma, field * (g.mapped ? 4 : (g.dim == 2 ? 3 : 6)) * g.nrhs, ctx->st));
  const long long full = (long long)g.n[0] * g.n[1] * g.n[2];
  const int blocks = (int)std::min<long long>((full + 255) / 256, 4096);
  const double h2 = ctx->h * ctx->h;
  if (g.mapped) {
    EWH_CU(alloc_zero(&w.met, field * 4, ctx->st));
    for (int k = 0; k < 4; ++k)
      to_padded_kernel<T><<<blocks, 256, 0, ctx->st>>>(g, d_met + (size_t)k * full, d_rho, 0, h2, w.met + k * field);
    ctx->launches += 4;
  }
  to_padded_kernel<T><<<blocks, 256, 0, ctx->st>>>(g, d_lam, d_rho, 0, h2, w.lam);
  to_padded_kernel<T><<<blocks, 256, 0, ctx->st>>>(g, d_mu, d_rho, 0, h2, w.mu);
  to_padded_kernel<T><<<blocks, 256, 0, ctx->st>>>(g, d_rho, d_rho, 1, h2, w.irh2);
  ctx->launches += 3;
  if (d_f) {
    EWH_CU(alloc_zero(&w.frho, state, ctx->st));
    for (int r = 0; r < g.nrhs; ++r)
      for (int c = 0; c < g.dim; ++c) {
        to_padded_kernel<T><<<blocks, 256, 0, ctx->st>>>(g, d_f + (size_t)(r * g.dim + c) * full, d_rho, 2, h2,
                                                         w.frho + (size_t)(r * g.dim + c) * field);
        ctx->launches += 1;
      }
  }
  EWH_CU(cudaGetLastError());
  if (sizeof(T) == 4 && g.dim == 2 && ctx->order == 4 && !g.mapped) {
    const int N = ctx->nt * ctx->periods;
    std::vector<double> hc(N), hw(N);
    for (int n = 0; n < N; ++n) {  // the same values as the per-level launches get
      hc[n] = std::cos(2.0 * M_PI * (double)(n % ctx->nt) / (double)ctx->nt);
      hw[n] = ctx->weights[n + 1];
    }
    EWH_CU(cudaMalloc(&w.d_cosn, sizeof(double) * N));
    EWH_CU(cudaMalloc(&w.d_wnew, sizeof(double) * N));
    EWH_CU(alloc_zero(&w.bar, RS_BAR_WORDS, ctx->st));
    const unsigned long long wait_ns = RS_WAIT_NS_DEFAULT;
    EWH_CU(cudaStreamSynchronize(ctx->st));
    EWH_CU(cudaMemcpy(w.bar + 2, &wait_ns, sizeof(wait_ns), cudaMemcpyHostToDevice));
    EWH_CU(cudaMemcpy(w.d_cosn, hc.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
    EWH_CU(cudaMemcpy(w.d_wnew, hw.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
    for (int k = 0; k < RS_SHAPES; ++k) w.rplan[k] = plan_resident_o4(g, k);
  }
  if (sizeof(T) == 4 && ctx->order == 4 && !g.mapped) {  // marching steps: 3D z-march, 2D y-march
    if (!w.bar) {
      EWH_CU(alloc_zero(&w.bar, RS_BAR_WORDS, ctx->st));
      const unsigned long long wait_ns = RS_WAIT_NS_DEFAULT;
      EWH_CU(cudaStreamSynchronize(ctx->st));
      EWH_CU(cudaMemcpy(w.bar + 2, &wait_ns, sizeof(wait_ns), cudaMemcpyHostToDevice));
    }
    w.zm = g.dim == 3 ? plan_zmarch(g, (const float*)w.u_a, (const float*)w.u_b, w.bar)
                      : plan_ymarch(g, (const float*)w.u_a, (const float*)w.u_b, w.bar);
  }
  return EWH_OK;
}

template <typename T>
void free_wave(Wave<T>& w) {
  if (w.cg_loop) cudaGraphExecDestroy(w.cg_loop);
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
  cudaFree(w.met);
  cudaFree(w.d_cosn);
  cudaFree(w.d_wnew);
  cudaFree(w.bar);
  w = Wave<T>();
}

template <typename T>
Wave<T>& wave_of(ewh_ctx* c);
template <>
Wave<double>& wave_of<double>(ewh_ctx* c) { return c->w64; }
template <>
Wave<float>& wave_of<float>(ewh_ctx* c) { return c->w32; }

// ---------------------------------------------------------------------------
// Autotuner: pick the step-kernel variant of a context by timing.
//
// The candidates (split or fused order-4 2D kernel; tile height of the
// order-2 2D kernel) are timed on the context's own buffers with 2 warm-up and
// 8 timed leapfrog levels each; the fastest wins.  Results are kept in a JSON
// file ($EWH_TUNE_CACHE, else $HOME/.cache/ewh/tune.json) keyed by the GPU and
// the problem's shape, so a shape is timed once per machine.  EWH_AUTOTUNE=0
// disables timing (variant 0).
// ---------------------------------------------------------------------------
std::string tune_cache_path() {
  const char* e = getenv("EWH_TUNE_CACHE");
  if (e && e[0]) return e;
  const char* h = getenv("HOME");
  if (!h || !h[0]) return "";
  return std::string(h) + "/.cache/ewh/tune.json";
}

std::vector<std::pair<std::string, int>> read_tune_cache(const std::string& path) {
  std::vector<std::pair<std::string, int>> out;
  FILE* f = path.empty() ? nullptr : fopen(path.c_str(), "r");
  if (!f) return out;
  char line[1024];
  while (fgets(line, sizeof line, f)) {
    char* q1 = strchr(line, '"');
    if (!q1) continue;
    char* q2 = strchr(q1 + 1, '"');
    if (!q2) continue;
    char* colon = strchr(q2, ':');
    if (!colon) continue;
    out.emplace_back(std::string(q1 + 1, q2), atoi(colon + 1));
  }
  fclose(f);
  return out;
}

void write_tune_cache(const std::string& path, const std::vector<std::pair<std::string, int>>& kv) {
  if (path.empty()) return;
  const size_t slash = path.find_last_of('/');
  if (slash != std::string::npos) {
    std::string dir = path.substr(0, slash);
    for (size_t i = 1; i <= dir.size(); ++i)
      if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);
  }
  const std::string tmp = path + ".tmp" + std::to_string((long long)getpid());
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return;
  fprintf(f, "{\n");
  for (size_t i = 0; i < kv.size(); ++i)
    fprintf(f, "  \"%s\": %d%s\n", kv[i].first.c_str(), kv[i].second, i + 1 < kv.size() ? "," : "");
  fprintf(f, "}\n");
  fclose(f);
  rename(tmp.c_str(), path.c_str());
}

template <typename T>
std::string tune_key(const ewh_ctx* ctx) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  std::string name = "gpu";
  if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
    name = prop.name;
    name += "-sm" + std::to_string(prop.major) + std::to_string(prop.minor) + "x" +
            std::to_string(prop.multiProcessorCount);
  } else {
    cudaGetLastError();
  }
  for (auto& ch : name)
    if (ch == '"' || ch == ' ') ch = '_';
  const Geom& g = ctx->g;
  // a batch member whose on-chip plans the batch rule excludes (resident_ok)
  // has other candidates than the same problem alone
  bool restricted = false;
  if (sizeof(T) == 4 && ctx->batch_member)
    for (int k = 0; k < RS_SHAPES; ++k)
      restricted = restricted || (ctx->w32.rplan[k].ok && (long long)ctx->w32.rplan[k].bx * ctx->w32.rplan[k].by <
                                                              RS_BATCH_MIN_BLOCK);
  return name + "|v4" + (restricted ? "b" : "") + (g.mapped ? "|map" : "") + "|d" + std::to_string(g.dim) +
         "|o" + std::to_string(ctx->order) + "|" +
         (sizeof(T) == 8 ? "f64" : "f32") + "|" + std::to_string(g.n[0]) + "x" + std::to_string(g.n[1]) + "x" +
         std::to_string(g.n[2]) + "|r" + std::to_string(g.nrhs);
}

// Resident variant v usable by this context?  (FP32 2D order 4, a
// partition that fits on chip, EWH_RESIDENT != 0.)
template <typename T>
bool resident_ok(const ewh_ctx* ctx, const Wave<T>& w, int v, bool named = false) {
  if (sizeof(T) != 4 || !is_resident_variant(v)) return false;
  const char* e = getenv("EWH_RESIDENT");
  if (e && e[0] == '0') return false;
  const ResidentPlan& p = w.rplan[v - VARIANT_RESIDENT];
  if (!p.ok) return false;
  // A batch runs its members' cooperative launches one after another, so a
  // member goes on chip only when its blocks are large enough that its own
  // launches keep the GPU busy; smaller members run their per-level kernels
  // in concurrent branches.  (EWH_STEP2D_O4=r<k> names the shape regardless.)
  if (ctx->batch_member && !named && (long long)p.bx * p.by < RS_BATCH_MIN_BLOCK) return false;
  return true;
}

// One cooperative launch running nsteps levels of the wave solve on chip.
template <typename T>
cudaError_t enqueue_resident(ewh_ctx* ctx, Wave<T>& w, int v, bool forced, int nsteps) {
  if constexpr (std::is_same<T, float>::value) {
    ResidentIO io{};
    io.u0 = w.u_a;
    io.xbuf0 = w.u_b;
    io.xbuf1 = w.delta;
    io.acc = w.acc;
    io.lam = w.lam;
    io.mu = w.mu;
    io.irh2 = w.irh2;
    io.frho = forced ? w.frho : nullptr;
    io.cosn = w.d_cosn;
    io.wnew = w.d_wnew;
    io.kt = ctx->kt;
    io.w0 = ctx->weights[0];
    io.nsteps = nsteps;
    io.bar = w.bar;
    return launch_resident_o4(ctx->g, w.rplan[v - VARIANT_RESIDENT], io, ctx->st);
  } else {
    (void)ctx;
    (void)w;
    (void)v;
    (void)forced;
    (void)nsteps;
    return cudaErrorInvalidValue;
  }
}

// The 2D order-4 FP32 y-march usable by this context?
template <typename T>
bool ymarch_ok(const ewh_ctx* ctx, const Wave<T>& w) {
  return sizeof(T) == 4 && ctx->g.dim == 2 && ctx->order == 4 && !ctx->g.mapped && w.zm.ok[0] != 0;
}

template <typename T>
void autotune(ewh_ctx* ctx, Wave<T>& w) {
  const int nbase = ctx->g.mapped ? 3 : step_variant_count(ctx->g.dim, ctx->order);
  const char* force = getenv("EWH_STEP2D_O4");
  // a launcher named by the environment (the y-march exists in FP32 only)
  const bool forced_launcher = force && (force[0] == 's' || force[0] == 'f' || (force[0] == 'y' && sizeof(T) == 4));
  bool any_res = false;
  for (int k = 0; k < RS_SHAPES && !forced_launcher; ++k) any_res |= resident_ok<T>(ctx, w, VARIANT_RESIDENT + k);
  const bool ym = ymarch_ok<T>(ctx, w) && !forced_launcher;
  // candidates: the launcher's own variants [0, nbase), the resident shapes,
  // the y-march (only the launcher's own when the environment names one)
  const int nv = ym ? YM_VARIANT + 1 : (any_res ? VARIANT_RESIDENT + RS_SHAPES : nbase);
  w.fallback = 0;
  if (force && force[0] == 'r') {  // EWH_STEP2D_O4=r, r0, r1, r2: resident solve of that CTA shape
    const int k = (force[1] >= '0' && force[1] < '0' + RS_SHAPES) ? force[1] - '0' : 0;
    if (resident_ok<T>(ctx, w, VARIANT_RESIDENT + k, true)) {
      w.variant = VARIANT_RESIDENT + k;
      return;
    }
  }
  if (force && strcmp(force, "ym") == 0 && ymarch_ok<T>(ctx, w)) {  // EWH_STEP2D_O4=ym: the y-march
    w.variant = YM_VARIANT;
    return;
  }
  const char* off = getenv("EWH_AUTOTUNE");
  if (nv <= 1 || (off && off[0] == '0')) {
    w.variant = 0;
    return;
  }
  // a choice made under EWH_STEP2D_O4 (a restricted candidate set) is cached
  // under its own key, so contexts of the same problem make the same choice
  const std::string path = tune_cache_path();
  std::string key = tune_key<T>(ctx);
  if (forced_launcher) {
    key += "|E";
    for (const char* c = force; *c; ++c)
      if (isalnum((unsigned char)*c)) key += *c;  // the cache file quotes keys as they are
  }
  auto cache = read_tune_cache(path);
  for (auto& kv : cache)
    if (kv.first == key && kv.second >= 0 && kv.second < nv &&
        (kv.second < nbase || (any_res && resident_ok<T>(ctx, w, kv.second)) || (kv.second == YM_VARIANT && ym))) {
      w.variant = kv.second;
      return;
    }
  WaveFields<T> f{};
  f.u_cur = w.u_a;
  f.u_next = w.u_b;
  f.delta = w.delta;
  f.acc = w.acc;
  f.lam = w.lam;
  f.mu = w.mu;
  f.irh2 = w.irh2;
  f.frho = nullptr;
  f.sigma = w.sigma;
  f.met = w.met;
  f.zm = &w.zm;
  StepScalars sc{ctx->kt, 1.0, 0.0, 0.0};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    w.variant = 0;
    return;
  }
  int best = 0, best_base = 0;
  float best_ms = 1e30f, best_base_ms = 1e30f;
  const int N = ctx->nt * ctx->periods;
  for (int v = 0; v < nv; ++v) {
    float per_level = 1e30f;
    if (is_resident_variant(v)) {
      if (any_res && resident_ok<T>(ctx, w, v)) {  // not when the environment names a per-level launcher
        const int ns = std::min(N, 40);
        bool ok = enqueue_resident<T>(ctx, w, v, false, std::min(N, 8)) == cudaSuccess;  // warm-up
        cudaEventRecord(e0, ctx->st);
        ok = ok && enqueue_resident<T>(ctx, w, v, false, ns) == cudaSuccess;
        cudaEventRecord(e1, ctx->st);
        float ms = 1e30f;
        if (ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
          per_level = ms / ns;
        cudaGetLastError();
      }
    } else if (v < nbase || (v == YM_VARIANT && ym)) {
      Geom g = ctx->g;
      g.variant = v;
      bool ok = true;
      for (int k = 0; k < 10 && ok; ++k) {
        if (k == 2) cudaEventRecord(e0, ctx->st);
        ok = launch_step<T>(g, ctx->order, f, STEP_MID, sc, ctx->st, nullptr) == cudaSuccess;
        std::swap(f.u_cur, f.u_next);
      }
      cudaEventRecord(e1, ctx->st);
      float ms = 1e30f;
      if (ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
        per_level = ms / 8;
      cudaGetLastError();
      if (per_level < best_base_ms) {
        best_base_ms = per_level;
        best_base = v;
      }
    }
    if (v <= YM_VARIANT) w.variant_ms[v] = per_level;
    if (per_level < best_ms) {
      best_ms = per_level;
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the timing levels wrote the state buffers: clear them back to zero
  const size_t state = (size_t)ctx->g.field * ctx->g.dim * ctx->g.nrhs;
  cudaMemsetAsync(w.u_a, 0, sizeof(T) * state, ctx->st);
  cudaMemsetAsync(w.u_b, 0, sizeof(T) * state, ctx->st);
  cudaMemsetAsync(w.delta, 0, sizeof(T) * state, ctx->st);
  cudaMemsetAsync(w.acc, 0, sizeof(T) * state, ctx->st);
  w.variant = best;
  w.fallback = best_base;
  if (getenv("EWH_VERBOSE")) {
    fprintf(stderr, "ewh: autotune %s:", key.c_str());
    for (int v = 0; v < nv && v <= YM_VARIANT; ++v) fprintf(stderr, " v%d=%.4g", v, w.variant_ms[v]);
    fprintf(stderr, " ms/level -> %d\n", best);
  }
  cache.emplace_back(key, best);
  write_tune_cache(path, cache);
}

// Enqueue the nt*periods steps of one wave solve (u^0 already in u_a).
template <typename T>
cudaError_t enqueue_steps(ewh_ctx* ctx, Wave<T>& w, bool forced, long long* nl) {
  const int N = ctx->nt * ctx->periods;
  if (is_resident_variant(w.variant)) {  // all levels in one cooperative launch per group of rhs
    cudaError_t e = enqueue_resident<T>(ctx, w, w.variant, forced, N);
    if (e == cudaSuccess && nl) *nl += w.rplan[w.variant - VARIANT_RESIDENT].groups;
    return e;
  }
  Geom gv = ctx->g;
  gv.variant = w.variant < 0 ? 0 : w.variant;
  WaveFields<T> f{};
  f.lam = w.lam;
  f.mu = w.mu;
  f.irh2 = w.irh2;
  f.frho = forced ? w.frho : nullptr;
  f.sigma = w.sigma;
  f.met = w.met;
  f.zm = &w.zm;
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
    cudaError_t e = launch_step<T>(gv, ctx->order, f, mode, s, ctx->st, nl);
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
  if (w.variant < 0) autotune<T>(ctx, w);
  for (int attempt = 0;; ++attempt) {
    cudaGraph_t graph = nullptr;
    EWH_CU(cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal));
    long long count = 0;
    cudaError_t e = enqueue_steps<T>(ctx, w, forced, &count);
    cudaError_t e2 = cudaStreamEndCapture(ctx->st, &graph);
    if (e == cudaSuccess && e2 == cudaSuccess) {
      e = cudaGraphInstantiate(&ge, graph, 0);
      e2 = cudaSuccess;
    }
    if (graph) cudaGraphDestroy(graph);
    if (e == cudaSuccess && e2 == cudaSuccess) {
      nk = count;
      return EWH_OK;
    }
    ge = nullptr;
    cudaGetLastError();
    if (attempt == 0 && is_resident_variant(w.variant)) {  // not capturable here: per-level launches
      w.variant = w.fallback;
      continue;
    }
    return fail(ctx, EWH_ECUDA, std::string("graph capture failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
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

// ---------------------------------------------------------------------------
// Implicit scheme (Section 4.4, eq. ImplicitScheme with the modified alpha
// and start), in mass form with B = I + (dt^2/2) M^{-1} K:
//   B u^{-1}  = (alpha/2) u^0 - (dt^2/2) (f/rho) cos(w dt),
//   B u^{n+1} = alpha u^n - B u^{n-1} - dt^2 (f/rho) cos(w t_n) cos(w dt),
// accumulated by the trapezoidal filter.  Each level solves with B by CG in
// the M inner product (B is M-self-adjoint and positive definite), started
// from the extrapolation 2 u^n - u^{n-1}, to a relative 1e-13.  FP64; the
// levels are host-driven (two synchronisations per inner iteration), so
// this path is not captured in graphs.
// ---------------------------------------------------------------------------
ewh_status mdot_dev(ewh_ctx* ctx, const double* x, const double* y, double* out_dev);
constexpr int I_RR = 0, I_PQ = 1, I_GG = 2, I_N = 3;

// dst = M^{-1} K src (dense FP64 vectors)
ewh_status implicit_minvK(ewh_ctx* ctx, const double* src, double* dst) {
  Wave<double>& w = ctx->w64;
  EWH_CU(launch_pack<double>(ctx->g, src, w.u_a, ctx->st));
  EWH_CU(launch_minvK<double>(ctx->g, ctx->order, w.u_a, w.u_b, w.lam, w.mu, w.irh2, w.sigma, ctx->st,
                              &ctx->launches, w.met));
  EWH_CU(launch_unpack<double>(ctx->g, w.u_b, dst, nullptr, ctx->st));
  ctx->launches += 2;
  return EWH_OK;
}

// dst = B src
ewh_status implicit_B(ewh_ctx* ctx, const double* src, double* dst) {
  ewh_status s = implicit_minvK(ctx, src, dst);
  if (s != EWH_OK) return s;
  EWH_CU(launch_axpby(total_unknowns(ctx), 1.0, src, 0.5 * ctx->dt * ctx->dt, dst, ctx->st));
  ctx->launches += 1;
  return EWH_OK;
}

// per-rhs M-dots into iscal[which][rhs], copied to the host
ewh_status implicit_dot(ewh_ctx* ctx, const double* x, const double* y, int which, std::vector<double>& out) {
  const int R = ctx->g.nrhs;
  ewh_status s = mdot_dev(ctx, x, y, ctx->iscal + (size_t)which * R);
  if (s != EWH_OK) return s;
  EWH_CU(cudaMemcpyAsync(out.data(), ctx->iscal + (size_t)which * R, sizeof(double) * R, cudaMemcpyDeviceToHost,
                         ctx->st));
  EWH_CU(cudaStreamSynchronize(ctx->st));
  return EWH_OK;
}

// Solve B x = g (x holds the starting guess) by CG in the M inner product.
ewh_status implicit_solve(ewh_ctx* ctx, const double* gv, double* x) {
  const int R = ctx->g.nrhs;
  const long long n = total_unknowns(ctx), seg = n / R;
  std::vector<double> rr(R), pq(R), gg(R), rr_new(R);
  ewh_status s = implicit_B(ctx, x, ctx->iq);
  if (s != EWH_OK) return s;
  EWH_CU(cudaMemcpyAsync(ctx->ir, gv, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->st));
  EWH_CU(launch_axpby(n, -1.0, ctx->iq, 1.0, ctx->ir, ctx->st));
  EWH_CU(cudaMemcpyAsync(ctx->ip, ctx->ir, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->st));
  s = implicit_dot(ctx, gv, gv, I_GG, gg);
  if (s != EWH_OK) return s;
  s = implicit_dot(ctx, ctx->ir, ctx->ir, I_RR, rr);
  if (s != EWH_OK) return s;
  const double tol2 = 1e-26;
  for (int it = 0;; ++it) {
    bool done = true;
    for (int k = 0; k < R; ++k) done = done && (rr[k] <= tol2 * gg[k]);
    if (done) return EWH_OK;
    if (it >= 5000) return fail(ctx, EWH_ENOTCONV, "implicit level: inner CG did not converge in 5000 iterations");
    s = implicit_B(ctx, ctx->ip, ctx->iq);
    if (s != EWH_OK) return s;
    s = implicit_dot(ctx, ctx->ip, ctx->iq, I_PQ, pq);
    if (s != EWH_OK) return s;
    for (int k = 0; k < R; ++k) {
      if (rr[k] <= tol2 * gg[k]) continue;
      if (!(pq[k] > 0.0)) return fail(ctx, EWH_EBREAKDOWN, "implicit level: inner CG lost definiteness");
      const double a = rr[k] / pq[k];
      EWH_CU(launch_axpby(seg, a, ctx->ip + k * seg, 1.0, x + k * seg, ctx->st));
      EWH_CU(launch_axpby(seg, -a, ctx->iq + k * seg, 1.0, ctx->ir + k * seg, ctx->st));
    }
    s = implicit_dot(ctx, ctx->ir, ctx->ir, I_RR, rr_new);
    if (s != EWH_OK) return s;
    for (int k = 0; k < R; ++k) {
      if (rr[k] <= tol2 * gg[k]) continue;
      EWH_CU(launch_axpby(seg, 1.0, ctx->ir + k * seg, rr_new[k] / rr[k], ctx->ip + k * seg, ctx->st));
      rr[k] = rr_new[k];
    }
    ++ctx->inner_iters;
  }
}

// acc = Pi u0 (forced) or S u0: all levels of the implicit scheme; u0 dense or
// null (zero).  The result is left in ctx->iacc.
ewh_status implicit_wave(ewh_ctx* ctx, const double* u0, bool forced) {
  const long long n = total_unknowns(ctx);
  const double dt = ctx->dt, c = 0.5 * dt * dt, cdt = std::cos(ctx->omega * dt);
  if (forced && !ctx->ifr) return fail(ctx, EWH_EINVAL, "problem was created without forcing");
  if (u0) EWH_CU(cudaMemcpyAsync(ctx->iu, u0, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->st));
  else EWH_CU(cudaMemsetAsync(ctx->iu, 0, sizeof(double) * n, ctx->st));
  // B u^{-1} = (alpha/2) u^0 - c (f/rho) cos(w dt); start from u^0
  EWH_CU(cudaMemsetAsync(ctx->ig, 0, sizeof(double) * n, ctx->st));
  EWH_CU(launch_axpby(n, 0.5 * ctx->alpha, ctx->iu, 0.0, ctx->ig, ctx->st));
  if (forced) EWH_CU(launch_axpby(n, -c * cdt, ctx->ifr, 1.0, ctx->ig, ctx->st));
  EWH_CU(cudaMemcpyAsync(ctx->iu_prev, ctx->iu, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->st));
  ewh_status s = implicit_solve(ctx, ctx->ig, ctx->iu_prev);
  if (s != EWH_OK) return s;
  // acc = w_0 u^0
  EWH_CU(cudaMemsetAsync(ctx->iacc, 0, sizeof(double) * n, ctx->st));
  EWH_CU(launch_axpby(n, ctx->weights[0], ctx->iu, 0.0, ctx->iacc, ctx->st));
  const int N = ctx->nt * ctx->periods;
  for (int lev = 0; lev < N; ++lev) {
    // g = alpha u^n - B u^{n-1} - dt^2 (f/rho) cos(w t_n) cos(w dt)
    s = implicit_B(ctx, ctx->iu_prev, ctx->ig);
    if (s != EWH_OK) return s;
    EWH_CU(launch_axpby(n, ctx->alpha, ctx->iu, -1.0, ctx->ig, ctx->st));
    if (forced) {
      const double cn = std::cos(2.0 * M_PI * (double)(lev % ctx->nt) / (double)ctx->nt);
      EWH_CU(launch_axpby(n, -dt * dt * cn * cdt, ctx->ifr, 1.0, ctx->ig, ctx->st));
    }
    // start from 2 u^n - u^{n-1}
    EWH_CU(cudaMemcpyAsync(ctx->iu_next, ctx->iu_prev, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->st));
    EWH_CU(launch_axpby(n, 2.0, ctx->iu, -1.0, ctx->iu_next, ctx->st));
    s = implicit_solve(ctx, ctx->ig, ctx->iu_next);
    if (s != EWH_OK) return s;
    double* t = ctx->iu_prev;
    ctx->iu_prev = ctx->iu;
    ctx->iu = ctx->iu_next;
    ctx->iu_next = t;
    EWH_CU(launch_axpby(n, ctx->weights[lev + 1], ctx->iu, 1.0, ctx->iacc, ctx->st));
    ctx->launches += 4;
  }
  return EWH_OK;
}

// v_out = S v_in (sub_from null) or sub_from - S v_in, implicit scheme
ewh_status implicit_S(ewh_ctx* ctx, const double* v_in, double* v_out, const double* sub_from) {
  const long long n = total_unknowns(ctx);
  ewh_status s = implicit_wave(ctx, v_in, false);
  if (s != EWH_OK) return s;
  if (sub_from) {
    if (sub_from != v_out) EWH_CU(cudaMemcpyAsync(v_out, sub_from, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->st));
    EWH_CU(launch_axpby(n, -1.0, ctx->iacc, 1.0, v_out, ctx->st));
  } else {
    EWH_CU(cudaMemcpyAsync(v_out, ctx->iacc, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->st));
  }
  return EWH_OK;
}

template <typename T>
ewh_status apply_S_T(ewh_ctx* ctx, const double* v_in, double* v_out, const double* sub_from) {
  if (ctx->implicit) return implicit_S(ctx, v_in, v_out, sub_from);
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
//
// The loop is split into cg_begin / cg_enqueue_iteration / cg_after_iteration
// so that a batch of problems can put the iterations of all its members into
// one graph and run the host-side logic per member afterwards.
struct CgState {
  double tol = 0.0, drop = 0.0;
  std::vector<double> anchor, true_res;
  bool any_active = false;
};

template <typename T>
ewh_status cg_begin(ewh_ctx* ctx, double* r, double tol, double drop, CgState& cs) {
  const int R = ctx->g.nrhs;
  const long long n = total_unknowns(ctx);
  ewh_status st = ctx->implicit ? EWH_OK : ensure_graph<T>(ctx, false);  // implicit: no step graph
  if (st != EWH_OK) return st;
  st = mdot_dev(ctx, r, r, sc(ctx, S_RR));
  if (st != EWH_OK) return st;
  EWH_CU(cudaMemsetAsync(ctx->kp, 0, sizeof(double) * n, ctx->st));
  EWH_CU(cudaMemsetAsync(sc(ctx, S_BETA), 0, sizeof(double) * R, ctx->st));
  EWH_CU(cudaMemsetAsync(ctx->flags, 0, sizeof(int), ctx->st));
  EWH_CU(cudaMemcpyAsync(ctx->h_scal, ctx->scal, sizeof(double) * S_N * R, cudaMemcpyDeviceToHost, ctx->st));
  EWH_CU(cudaStreamSynchronize(ctx->st));
  cs.tol = tol;
  cs.drop = drop;
  cs.anchor.assign(R, 0.0);
  cs.true_res.assign(R, 0.0);
  cs.any_active = false;
  double worst = 0.0;
  for (int k = 0; k < R; ++k) {
    cs.true_res[k] = std::sqrt(ctx->h_scal[S_RR * R + k] / ctx->h_scal[S_BB * R + k]);
    cs.anchor[k] = cs.true_res[k];
    ctx->h_act[k] = cs.true_res[k] > tol ? 1 : 0;
    cs.any_active = cs.any_active || ctx->h_act[k];
    worst = std::max(worst, cs.true_res[k]);
  }
  EWH_CU(cudaMemcpyAsync(ctx->active, ctx->h_act, sizeof(int) * R, cudaMemcpyHostToDevice, ctx->st));
  ctx->history.push_back(worst);
  return EWH_OK;
}

// Scalars, active mask and flags of the last iteration into pinned host memory.
cudaError_t copy_cg_scalars(ewh_ctx* ctx) {
  const int R = ctx->g.nrhs;
  cudaError_t e = cudaMemcpyAsync(ctx->h_scal, ctx->scal, sizeof(double) * S_N * R, cudaMemcpyDeviceToHost, ctx->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_act, ctx->active, sizeof(int) * R, cudaMemcpyDeviceToHost, ctx->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_flag, ctx->flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->st);
  return e;
}

// One CG iteration on ctx->st, ending (with `copies`) with the copies of the
// scalars, the active mask and the flags into pinned host memory.  With
// direct_steps the leapfrog launches are enqueued one by one (inside a batch
// or loop capture); otherwise the context's captured S graph is launched.
template <typename T>
ewh_status cg_enqueue_iteration(ewh_ctx* ctx, double* x, double* r, bool direct_steps, bool copies = true) {
  const Geom& g = ctx->g;
  const int R = g.nrhs;
  Wave<T>& w = wave_of<T>(ctx);
  // p = r + beta p ; u^0 = p
  EWH_CU(launch_pupdate_pack<T>(g, r, ctx->kp, sc(ctx, S_BETA), w.u_a, ctx->st));
  ctx->launches += 1;
  if (ctx->implicit) {  // q = p - S p by the implicit levels
    ewh_status s = implicit_S(ctx, ctx->kp, ctx->kq, ctx->kp);
    if (s != EWH_OK) return s;
  } else if (direct_steps) {
    long long count = 0;
    EWH_CU(enqueue_steps<T>(ctx, w, false, &count));
    ctx->launches += count;
  } else {
    EWH_CU(launch_timed_graph<T>(ctx, w.graph_S));
    ctx->launches += w.graph_S_kernels;
  }
  // q = p - S p
  if (!ctx->implicit) EWH_CU(launch_unpack<T>(g, w.acc, ctx->kq, ctx->kp, ctx->st));
  EWH_CU(launch_mdot_partial(g, ctx->mw, ctx->kp, ctx->kq, ctx->part, ctx->st));
  EWH_CU(launch_cg_alpha(R, ctx->part, ctx->nblk, sc(ctx, S_RR), sc(ctx, S_ALPHA), ctx->active, ctx->flags,
                         ctx->st));
  EWH_CU(launch_cg_xr_update(g, ctx->mw, sc(ctx, S_ALPHA), ctx->kp, ctx->kq, x, r, ctx->part, ctx->st));
  EWH_CU(launch_cg_beta(R, ctx->part, ctx->nblk, sc(ctx, S_RR), sc(ctx, S_BB), sc(ctx, S_BETA), sc(ctx, S_RES),
                        ctx->active, ctx->st));
  ctx->launches += 5;
  if (copies) EWH_CU(copy_cg_scalars(ctx));
  return EWH_OK;
}

// Host logic after an iteration whose copies have completed.
template <typename T>
ewh_status cg_after_iteration(ewh_ctx* ctx, double* x, double* r, CgState& cs, ewh_solve_info* inf) {
  const int R = ctx->g.nrhs;
  ++inf->iters;
  if (sizeof(T) == 8) ++inf->s_applies_fp64;
  else ++inf->s_applies;
  if (*ctx->h_flag & 1)
    return fail(ctx, EWH_EBREAKDOWN, "CG breakdown: (p, (I-S)p)_M <= 0 (indefinite system near resonance)");
  bool replace = false;
  double hist = 0.0;
  for (int k = 0; k < R; ++k) {
    const double res = ctx->h_scal[S_RES * R + k];
    if (ctx->h_act[k]) {
      hist = std::max(hist, res);
      if (res <= cs.tol || (cs.drop > 0.0 && res <= cs.drop * cs.anchor[k])) replace = true;
    }
  }
  ctx->history.push_back(hist);
  if (replace) {
    double dummy = 0.0;
    ewh_status st = true_residual(ctx, x, r, &dummy);
    if (st != EWH_OK) return st;
    ++inf->s_applies_fp64;
    EWH_CU(launch_cg_replace(R, sc(ctx, S_DOT), sc(ctx, S_RR), sc(ctx, S_BETA), sc(ctx, S_RES), sc(ctx, S_BB),
                             ctx->st));
    ctx->launches += 1;
    bool changed = false;
    for (int k = 0; k < R; ++k) {
      cs.true_res[k] = std::sqrt(ctx->h_scal[S_DOT * R + k] / ctx->h_scal[S_BB * R + k]);
      cs.anchor[k] = cs.true_res[k];
      if (ctx->h_act[k] && cs.true_res[k] <= cs.tol) {
        ctx->h_act[k] = 0;
        changed = true;
      }
    }
    if (changed) EWH_CU(cudaMemcpyAsync(ctx->active, ctx->h_act, sizeof(int) * R, cudaMemcpyHostToDevice, ctx->st));
  }
  cs.any_active = false;
  for (int k = 0; k < R; ++k) cs.any_active = cs.any_active || ctx->h_act[k];
  return EWH_OK;
}

double cg_worst_true(const CgState& cs) {
  double m = 0.0;
  for (double v : cs.true_res) m = std::max(m, v);
  return m;
}

// Iterations per host poll of the device-controlled CG loop (EWH_CG_POLL,
// default 32; 1 or less: the host drives every iteration).
int cg_window() {
  const char* e = getenv("EWH_CG_POLL");
  const int m = e ? atoi(e) : 32;
  return std::min(m, CG_WINDOW_MAX);
}

// Build the device-controlled CG loop of precision T on (ctx->kx, ctx->kr):
// a graph whose while-conditional node runs one iteration per pass (the
// leapfrog launches, the Krylov kernels, then cg_control, which sets the
// condition), so a window of iterations runs without the host.  Any failure
// (a launch the driver does not take inside a conditional body) leaves
// cg_loop_state = -1 and the host-driven loop in charge.
template <typename T>
void ensure_cg_loop(ewh_ctx* ctx) {
  Wave<T>& w = wave_of<T>(ctx);
  if (w.cg_loop_state != 0 || ctx->implicit) {
    if (ctx->implicit) w.cg_loop_state = -1;
    return;
  }
  w.cg_loop_state = -1;
  cudaGraph_t graph = nullptr;
  cudaGraphConditionalHandle h;
  if (cudaGraphCreate(&graph, 0) != cudaSuccess ||
      cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return;
  }
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  bool ok = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np) == cudaSuccess;
  if (ok) {
    cudaGraph_t body = np.conditional.phGraph_out[0];
    ok = cudaStreamBeginCaptureToGraph(ctx->st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
         cudaSuccess;
    if (ok) {
      const long long l0 = ctx->launches;
      ok = cg_enqueue_iteration<T>(ctx, ctx->kx, ctx->kr, true, false) == EWH_OK &&
           launch_cg_control(h, ctx->g.nrhs, sc(ctx, S_RES), ctx->active, ctx->d_anchor, ctx->flags, ctx->d_loop,
                             ctx->d_hist, ctx->st) == cudaSuccess;
      w.cg_loop_kernels = ctx->launches - l0 + 1;
      ctx->launches = l0;  // captured, not run
      cudaGraph_t captured = nullptr;
      ok = cudaStreamEndCapture(ctx->st, &captured) == cudaSuccess && ok;
    }
  }
  ok = ok && cudaGraphInstantiate(&w.cg_loop, graph, 0) == cudaSuccess;
  cudaGraphDestroy(graph);
  if (!ok) {
    if (w.cg_loop) cudaGraphExecDestroy(w.cg_loop);
    w.cg_loop = nullptr;
    cudaGetLastError();
    if (getenv("EWH_VERBOSE")) fprintf(stderr, "ewh: device-controlled CG loop unavailable: host polls each iteration\n");
    return;
  }
  w.cg_loop_state = 1;
}

template <typename T>
ewh_status run_cg(ewh_ctx* ctx, double* x, double* r, double tol, int maxit, double drop, ewh_solve_info* inf,
                  double* rel_out) {
  CgState cs;
  ewh_status st = cg_begin<T>(ctx, r, tol, drop, cs);
  if (st != EWH_OK) return st;
  const int R = ctx->g.nrhs;
  const int m = cg_window();
  Wave<T>& w = wave_of<T>(ctx);
  // the loop graph works on x = kx, r = kr; tol and drop follow the anchors
  if (m > 1 && x == ctx->kx && r == ctx->kr && w.cg_loop_state == 0) ensure_cg_loop<T>(ctx);
  const bool dev = m > 1 && x == ctx->kx && r == ctx->kr && w.cg_loop_state == 1;
  while (cs.any_active && inf->iters < maxit) {
    if (dev) {
      // a window of iterations under device control; the host then takes the
      // decisions of the window's last iteration (as after any iteration)
      const int limit = std::min(m, maxit - inf->iters);
      for (int k = 0; k < R; ++k) ctx->h_anchor[k] = cs.anchor[k];
      ctx->h_anchor[R] = tol;
      ctx->h_anchor[R + 1] = drop;
      ctx->h_loop[0] = 0;
      ctx->h_loop[1] = limit;
      EWH_CU(cudaMemcpyAsync(ctx->d_anchor, ctx->h_anchor, sizeof(double) * (R + 2), cudaMemcpyHostToDevice,
                             ctx->st));
      EWH_CU(cudaMemcpyAsync(ctx->d_loop, ctx->h_loop, sizeof(int) * 2, cudaMemcpyHostToDevice, ctx->st));
      EWH_CU(cudaGraphLaunch(w.cg_loop, ctx->st));
      EWH_CU(copy_cg_scalars(ctx));
      EWH_CU(cudaMemcpyAsync(ctx->h_loop, ctx->d_loop, sizeof(int) * 2, cudaMemcpyDeviceToHost, ctx->st));
      EWH_CU(cudaMemcpyAsync(ctx->h_hist, ctx->d_hist, sizeof(double) * limit, cudaMemcpyDeviceToHost, ctx->st));
      EWH_CU(cudaStreamSynchronize(ctx->st));
      const int it = ctx->h_loop[0];
      if (it < 1 || it > limit) return fail(ctx, EWH_ECUDA, "device-controlled CG loop ran no iteration");
      ctx->launches += (long long)it * w.cg_loop_kernels;
      ctx->loop_steps[sizeof(T) == 4 ? 1 : 0] += (long long)it * ctx->nt * ctx->periods;
      ctx->loop_waves[sizeof(T) == 4 ? 1 : 0] += it;
      for (int i = 0; i + 1 < it; ++i) {  // iterations that needed no host decision
        ctx->history.push_back(ctx->h_hist[i]);
        ++inf->iters;
        if (sizeof(T) == 8) ++inf->s_applies_fp64;
        else ++inf->s_applies;
      }
    } else {
      st = cg_enqueue_iteration<T>(ctx, x, r, false);
      if (st != EWH_OK) return st;
      EWH_CU(cudaStreamSynchronize(ctx->st));
    }
    st = cg_after_iteration<T>(ctx, x, r, cs, inf);
    if (st != EWH_OK) {
      *rel_out = cg_worst_true(cs);
      return st;
    }
  }
  *rel_out = cg_worst_true(cs);
  return EWH_OK;
}

// Conjugate residual in the M inner product (the paper's choice for its FD
// sweeps: the residual norm never increases).  On entry x is the iterate and
// r its true FP64 residual; one S apply (precision T) per iteration:
//   alpha = (r, Ar)/(Ap, Ap); x += alpha p; r -= alpha Ap; Ar = A r;
//   beta = (r, Ar)_new/(r, Ar)_old; p = r + beta p; Ap = Ar + beta Ap.
// When the recursive residual reaches tol (or, for FP32, falls tenfold since
// the last check) r is replaced by the FP64 true residual and the direction
// set restarts from it (p = r, Ap = A r); convergence is declared on the true
// residual only.
template <typename T>
ewh_status ar_apply(ewh_ctx* ctx, double* src, double* dst) {
  if (ctx->implicit) return implicit_S(ctx, src, dst, src);
  Wave<T>& w = wave_of<T>(ctx);
  EWH_CU(launch_pack<T>(ctx->g, src, w.u_a, ctx->st));
  EWH_CU(launch_timed_graph<T>(ctx, w.graph_S));
  EWH_CU(launch_unpack<T>(ctx->g, w.acc, dst, src, ctx->st));  // dst = src - S src
  ctx->launches += 2 + w.graph_S_kernels;
  return EWH_OK;
}

template <typename T>
ewh_status cr_restart(ewh_ctx* ctx, double* r, ewh_solve_info* inf) {
  const long long n = total_unknowns(ctx);
  ewh_status st = ar_apply<T>(ctx, r, ctx->kar);
  if (st != EWH_OK) return st;
  if (sizeof(T) == 8) ++inf->s_applies_fp64;
  else ++inf->s_applies;
  EWH_CU(cudaMemcpyAsync(ctx->kp, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->st));
  EWH_CU(cudaMemcpyAsync(ctx->kap, ctx->kar, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->st));
  EWH_CU(launch_mdot_partial(ctx->g, ctx->mw, r, ctx->kar, ctx->part, ctx->st));
  EWH_CU(launch_cr_beta(ctx->g.nrhs, ctx->part, ctx->nblk, sc(ctx, S_DOT), sc(ctx, S_BETA), ctx->active, 1, ctx->st));
  ctx->launches += 2;
  return EWH_OK;
}

template <typename T>
ewh_status run_cr(ewh_ctx* ctx, double* x, double* r, double tol, int maxit, double drop, ewh_solve_info* inf,
                  double* rel_out) {
  const Geom& g = ctx->g;
  const int R = g.nrhs;
  ewh_status st = ctx->implicit ? EWH_OK : ensure_graph<T>(ctx, false);  // implicit: no step graph
  if (st != EWH_OK) return st;
  // true residual norms and active mask
  st = mdot_dev(ctx, r, r, sc(ctx, S_RR));
  if (st != EWH_OK) return st;
  EWH_CU(cudaMemsetAsync(ctx->flags, 0, sizeof(int), ctx->st));
  EWH_CU(cudaMemcpyAsync(ctx->h_scal, ctx->scal, sizeof(double) * S_N * R, cudaMemcpyDeviceToHost, ctx->st));
  EWH_CU(cudaStreamSynchronize(ctx->st));
  std::vector<double> true_res(R), anchor(R);
  bool any = false;
  for (int k = 0; k < R; ++k) {
    true_res[k] = anchor[k] = std::sqrt(ctx->h_scal[S_RR * R + k] / ctx->h_scal[S_BB * R + k]);
    ctx->h_act[k] = true_res[k] > tol;
    any = any || ctx->h_act[k];
  }
  EWH_CU(cudaMemcpyAsync(ctx->active, ctx->h_act, sizeof(int) * R, cudaMemcpyHostToDevice, ctx->st));
  auto worst = [&]() {
    double m = 0.0;
    for (double v : true_res) m = std::max(m, v);
    return m;
  };
  ctx->history.push_back(worst());
  if (any) {
    st = cr_restart<T>(ctx, r, inf);
    if (st != EWH_OK) return st;
  }
  while (any && inf->iters < maxit) {
    // alpha = (r, Ar) / (Ap, Ap)      (S_DOT holds (r, Ar))
    EWH_CU(launch_mdot_partial(g, ctx->mw, ctx->kap, ctx->kap, ctx->part, ctx->st));
    EWH_CU(launch_cg_alpha(R, ctx->part, ctx->nblk, sc(ctx, S_DOT), sc(ctx, S_ALPHA), ctx->active, ctx->flags,
                           ctx->st));
    // x += alpha p ; r -= alpha Ap ; res = ||r||_M / ||b||_M
    EWH_CU(launch_cg_xr_update(g, ctx->mw, sc(ctx, S_ALPHA), ctx->kp, ctx->kap, x, r, ctx->part, ctx->st));
    EWH_CU(launch_res(R, ctx->part, ctx->nblk, sc(ctx, S_BB), sc(ctx, S_RES), ctx->active, ctx->st));
    ctx->launches += 4;
    // Ar = A r ; beta ; p, Ap
    st = ar_apply<T>(ctx, r, ctx->kar);
    if (st != EWH_OK) return st;
    EWH_CU(launch_mdot_partial(g, ctx->mw, r, ctx->kar, ctx->part, ctx->st));
    EWH_CU(launch_cr_beta(R, ctx->part, ctx->nblk, sc(ctx, S_DOT), sc(ctx, S_BETA), ctx->active, 0, ctx->st));
    EWH_CU(launch_cr_pupdate(g, r, ctx->kar, ctx->kp, ctx->kap, sc(ctx, S_BETA), ctx->st));
    ctx->launches += 3;
    ++inf->iters;
    if (sizeof(T) == 8) ++inf->s_applies_fp64;
    else ++inf->s_applies;
    EWH_CU(cudaMemcpyAsync(ctx->h_scal, ctx->scal, sizeof(double) * S_N * R, cudaMemcpyDeviceToHost, ctx->st));
    EWH_CU(cudaMemcpyAsync(ctx->h_flag, ctx->flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    EWH_CU(cudaStreamSynchronize(ctx->st));
    if (*ctx->h_flag & 1) {
      *rel_out = worst();
      return fail(ctx, EWH_EBREAKDOWN, "CR breakdown: (Ap, Ap)_M <= 0");
    }
    bool replace = false;
    double hist = 0.0;
    for (int k = 0; k < R; ++k) {
      if (!ctx->h_act[k]) continue;
      const double res = ctx->h_scal[S_RES * R + k];
      hist = std::max(hist, res);
      if (res <= tol || (drop > 0.0 && res <= drop * anchor[k])) replace = true;
    }
    ctx->history.push_back(hist);
    if (replace) {
      double dummy = 0.0;
      st = true_residual(ctx, x, r, &dummy);
      if (st != EWH_OK) return st;
      ++inf->s_applies_fp64;
      bool changed = false;
      any = false;
      for (int k = 0; k < R; ++k) {
        true_res[k] = anchor[k] = std::sqrt(ctx->h_scal[S_DOT * R + k] / ctx->h_scal[S_BB * R + k]);
        if (ctx->h_act[k] && true_res[k] <= tol) {
          ctx->h_act[k] = 0;
          changed = true;
        }
        any = any || ctx->h_act[k];
      }
      if (changed) EWH_CU(cudaMemcpyAsync(ctx->active, ctx->h_act, sizeof(int) * R, cudaMemcpyHostToDevice, ctx->st));
      if (any) {
        st = cr_restart<T>(ctx, r, inf);
        if (st != EWH_OK) return st;
      }
    }
  }
  *rel_out = worst();
  return EWH_OK;
}

// MINRES in the M inner product (Section 4.4, the remark on the implicit
// scheme: with few quadrature points near a resonance the discrete filter
// transfer function can exceed 1 and M(I - S) become indefinite; MINRES then
// replaces CG).  Lanczos in the M inner product builds T_k; Givens rotations
// factor it, and the iterate minimising ||b - A x||_M over x0 + K_k follows
// from the direction recurrence w_k = (v_k - rho2 w_{k-1} - rho3 w_{k-2})/rho1.
// One S apply (precision T) per iteration; the right-hand sides advance
// together, each with its own Lanczos and rotation scalars (host, FP64).  When
// the recursive residual |eta| reaches tol (or, for FP32, falls by `drop`
// since the last check, or the Krylov space is exhausted) the FP64 true
// residual replaces it and the recurrence restarts from the current iterate;
// convergence is declared on the true residual only.
template <typename T>
ewh_status run_minres(ewh_ctx* ctx, double* x, double* r, double tol, int maxit, double drop, ewh_solve_info* inf,
                      double* rel_out) {
  const Geom& g = ctx->g;
  const int R = g.nrhs;
  const long long n = total_unknowns(ctx);
  const long long seg = n / R;  // unknowns of one right-hand side
  ewh_status st = ctx->implicit ? EWH_OK : ensure_graph<T>(ctx, false);  // implicit: no step graph
  if (st != EWH_OK) return st;
  double* v_prev = ctx->kp;
  double* v = ctx->kq;
  double* z = ctx->kar;
  double* w1 = ctx->kap;  // w_{k-1}
  double* w2 = ctx->kd;   // w_{k-2}, overwritten by w_k
  std::vector<double> bnorm(R), beta(R), eta(R), c1(R), s1(R), c2(R), s2(R), true_res(R), anchor(R), alpha(R),
      beta_next(R);
  std::vector<char> act(R, 0);
  auto fetch = [&](int which, std::vector<double>& out) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(ctx->h_scal, ctx->scal, sizeof(double) * S_N * R, cudaMemcpyDeviceToHost, ctx->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
    for (int k = 0; k < R; ++k) out[k] = ctx->h_scal[which * R + k];
    return e;
  };
  {
    std::vector<double> bb(R);
    EWH_CU(fetch(S_BB, bb));
    for (int k = 0; k < R; ++k) bnorm[k] = std::sqrt(bb[k]);
  }
  // (re)start from the true residual r of x: v = r / ||r||_M
  auto restart = [&](bool first) -> ewh_status {
    ewh_status e2 = mdot_dev(ctx, r, r, sc(ctx, S_DOT));
    if (e2 != EWH_OK) return e2;
    std::vector<double> rr(R);
    EWH_CU(fetch(S_DOT, rr));
    EWH_CU(cudaMemsetAsync(v, 0, sizeof(double) * n, ctx->st));
    EWH_CU(cudaMemsetAsync(v_prev, 0, sizeof(double) * n, ctx->st));
    EWH_CU(cudaMemsetAsync(w1, 0, sizeof(double) * n, ctx->st));
    EWH_CU(cudaMemsetAsync(w2, 0, sizeof(double) * n, ctx->st));
    for (int k = 0; k < R; ++k) {
      beta[k] = std::sqrt(rr[k]);
      true_res[k] = anchor[k] = beta[k] / bnorm[k];
      if (first) act[k] = true_res[k] > tol;
      else act[k] = act[k] && true_res[k] > tol;
      c1[k] = c2[k] = 1.0;
      s1[k] = s2[k] = 0.0;
      eta[k] = beta[k];
      if (act[k]) {
        EWH_CU(launch_axpby(seg, 1.0 / beta[k], r + k * seg, 1.0, v + k * seg, ctx->st));
        ctx->launches += 1;
      }
    }
    return EWH_OK;
  };
  auto worst = [&]() {
    double m = 0.0;
    for (double t : true_res) m = std::max(m, t);
    return m;
  };
  st = restart(true);
  if (st != EWH_OK) return st;
  ctx->history.push_back(worst());
  auto any_active = [&]() {
    for (char a : act)
      if (a) return true;
    return false;
  };
  while (any_active() && inf->iters < maxit) {
    // Lanczos: z = A v - beta_k v_{k-1}; alpha = (v, z)_M; z -= alpha v; beta_{k+1} = ||z||_M
    st = ar_apply<T>(ctx, v, z);
    if (st != EWH_OK) return st;
    for (int k = 0; k < R; ++k)
      if (act[k]) EWH_CU(launch_axpby(seg, -beta[k], v_prev + k * seg, 1.0, z + k * seg, ctx->st));
    st = mdot_dev(ctx, v, z, sc(ctx, S_DOT));
    if (st != EWH_OK) return st;
    EWH_CU(fetch(S_DOT, alpha));
    for (int k = 0; k < R; ++k)
      if (act[k]) EWH_CU(launch_axpby(seg, -alpha[k], v + k * seg, 1.0, z + k * seg, ctx->st));
    st = mdot_dev(ctx, z, z, sc(ctx, S_DOT));
    if (st != EWH_OK) return st;
    EWH_CU(fetch(S_DOT, beta_next));
    ++inf->iters;
    if (sizeof(T) == 8) ++inf->s_applies_fp64;
    else ++inf->s_applies;
    bool check = false;
    double hist = 0.0;
    for (int k = 0; k < R; ++k) {
      if (!act[k]) continue;
      const double bn = std::sqrt(std::max(beta_next[k], 0.0));
      // the two previous rotations act on the new column (0, beta_k, alpha_k, beta_{k+1})
      const double rho3 = s2[k] * beta[k];
      const double tt = c2[k] * beta[k];
      const double rho2 = c1[k] * tt + s1[k] * alpha[k];
      const double delta = -s1[k] * tt + c1[k] * alpha[k];
      const double rho1 = std::hypot(delta, bn);
      if (!(rho1 > 0.0) || !std::isfinite(rho1)) {
        *rel_out = worst();
        return fail(ctx, EWH_EBREAKDOWN, "MINRES breakdown: singular or non-finite tridiagonal");
      }
      const double c = delta / rho1, sn = bn / rho1;
      // w_k = (v_k - rho2 w_{k-1} - rho3 w_{k-2}) / rho1 (into the w_{k-2} buffer); x += c eta w_k
      EWH_CU(launch_axpby(seg, -rho2 / rho1, w1 + k * seg, -rho3 / rho1, w2 + k * seg, ctx->st));
      EWH_CU(launch_axpby(seg, 1.0 / rho1, v + k * seg, 1.0, w2 + k * seg, ctx->st));
      EWH_CU(launch_axpby(seg, c * eta[k], w2 + k * seg, 1.0, x + k * seg, ctx->st));
      // v_{k+1} = z / beta_{k+1} (in place in z)
      if (bn > 0.0) EWH_CU(launch_axpby(seg, 0.0, z + k * seg, 1.0 / bn, z + k * seg, ctx->st));
      ctx->launches += 6;
      eta[k] = -sn * eta[k];
      c2[k] = c1[k];
      s2[k] = s1[k];
      c1[k] = c;
      s1[k] = sn;
      beta[k] = bn;
      const double res = std::fabs(eta[k]) / bnorm[k];
      hist = std::max(hist, res);
      if (res <= tol || (drop > 0.0 && res <= drop * anchor[k]) || bn == 0.0) check = true;
    }
    ctx->launches += 4;
    ctx->history.push_back(hist);
    // rotate buffers: (v_prev, v, z) <- (v, z, v_prev); (w1, w2) <- (w_k, w_{k-1})
    std::swap(w1, w2);
    double* tmp = v_prev;
    v_prev = v;
    v = z;
    z = tmp;
    if (check) {
      double dummy = 0.0;
      st = true_residual(ctx, x, r, &dummy);
      if (st != EWH_OK) return st;
      ++inf->s_applies_fp64;
      st = restart(false);
      if (st != EWH_OK) return st;
    }
  }
  *rel_out = worst();
  return EWH_OK;
}

// CG met (p, A p)_M <= 0 on the FP64 operator: M(I - S) is indefinite, or
// numerically so next to a resonance.  Continue from the current iterate with
// MINRES (the remark of Section 4.4 on indefinite systems), restarted from the
// true FP64 residual; its iterations are counted in inf->minres_iters.
// *result becomes MINRES's status.
ewh_status minres_after_breakdown(ewh_ctx* ctx, double tol, int maxit, ewh_solve_info* inf, double* rel,
                                  ewh_status* result) {
  ewh_status s = true_residual(ctx, ctx->kx, ctx->kr, rel);
  if (s != EWH_OK) return s;
  ++inf->s_applies_fp64;
  ctx->err = "no error";
  const int it0 = inf->iters;
  *result = run_minres<double>(ctx, ctx->kx, ctx->kr, tol, maxit, 0.0, inf, rel);
  inf->minres_iters += inf->iters - it0;
  return EWH_OK;
}

ewh_status solve_impl(ewh_ctx* ctx, double tol, int maxit, const double* x0, double* v_out,
                      ewh_solve_info* inf, int method = 0) {
  const Geom& g = ctx->g;
  const long long n = total_unknowns(ctx);
  ctx->history.clear();
  // b = Pi 0 in FP64: the right-hand side every residual is measured against
  ewh_status s = EWH_OK;
  if (ctx->implicit) {
    s = implicit_wave(ctx, nullptr, true);
    if (s != EWH_OK) return s;
    EWH_CU(cudaMemcpyAsync(ctx->kb, ctx->iacc, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->st));
  } else {
    s = run_wave<double>(ctx, nullptr, true);
    if (s != EWH_OK) return s;
    EWH_CU(launch_unpack<double>(g, ctx->w64.acc, ctx->kb, nullptr, ctx->st));
  }
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
  if (method == 2) {
    result = ctx->precision == EWH_FP64 ? run_minres<double>(ctx, ctx->kx, ctx->kr, tol, maxit, 0.0, inf, &rel)
                                        : run_minres<float>(ctx, ctx->kx, ctx->kr, tol, maxit, 0.1, inf, &rel);
  } else if (method == 1) {
    result = ctx->precision == EWH_FP64 ? run_cr<double>(ctx, ctx->kx, ctx->kr, tol, maxit, 0.0, inf, &rel)
                                        : run_cr<float>(ctx, ctx->kx, ctx->kr, tol, maxit, 0.1, inf, &rel);
  } else if (ctx->precision == EWH_FP64) {
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
  if (result == EWH_EBREAKDOWN && method != 2) {  // CG or CR met an indefinite system
    s = minres_after_breakdown(ctx, tol, maxit, inf, &rel, &result);
    if (s != EWH_OK) return s;
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
  {  // one padded component must index in 32 bits (the step kernels use int offsets)
    long long cells = 1;
    for (int a = 0; a < d->dim; ++a)
      cells *= ((d->n[a] + TILE_ROUND - 1) / TILE_ROUND) * TILE_ROUND + (a == 0 ? PAD3X : 2 * PAD);
    if (cells >= (1LL << 31)) return fail(nullptr, EWH_EINVAL, "grid too large: a padded component must hold < 2^31 nodes");
  }
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
  if (d->implicit != 0 && d->implicit != 1) return fail(nullptr, EWH_EINVAL, "implicit must be 0 or 1");
  if (d->implicit && (d->precision != EWH_FP64 || d->nt < 5))
    return fail(nullptr, EWH_EINVAL, "the implicit scheme needs precision EWH_FP64 and an explicit nt >= 5");
  return EWH_OK;
}

}  // namespace

struct ewh_batch {
  std::vector<ewh_ctx*> p;
  cudaStream_t user_stream = nullptr;
  cudaStream_t master = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins;
  cudaGraphExec_t iter_graph = nullptr;
  std::vector<int> graph_members;
  // CG windows under device control: one while-conditional node per member
  cudaGraphExec_t loop_graph = nullptr;
  std::vector<int> loop_members;
  std::vector<long long> loop_kernels;  // per member: kernels of one pass
  bool loop_failed = false;
  int precision = EWH_FP64;
  long long launches = 0;
  std::string err = "no error";
};

namespace {

ewh_status bfail(ewh_batch* b, ewh_status s, const std::string& m) {
  b->err = m;
  return s;
}

// Capture one graph whose branches enqueue `fn(k)` on member k's stream.
// The branches run concurrently, except when a member runs the resident
// solve: a cooperative launch must have its whole grid resident, so then the
// members follow one another.
template <typename F>
ewh_status capture_branches(ewh_batch* b, const std::vector<int>& members, F fn, cudaGraphExec_t* out) {
  bool serial = false;
  if (b->precision != EWH_FP64)
    for (int k : members) serial = serial || is_resident_variant(b->p[k]->w32.variant);
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(b->master, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return bfail(b, EWH_ECUDA, "batch capture could not start");
  cudaError_t e = cudaEventRecord(b->fork, b->master);
  ewh_status st = EWH_OK;
  cudaEvent_t prev = b->fork;
  for (int k : members) {
    ewh_ctx* c = b->p[k];
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->st, serial ? prev : b->fork, 0);
    if (e == cudaSuccess && st == EWH_OK) st = fn(k);
    if (e == cudaSuccess) e = cudaEventRecord(b->joins[k], c->st);
    if (e == cudaSuccess && !serial) e = cudaStreamWaitEvent(b->master, b->joins[k], 0);
    prev = b->joins[k];
  }
  if (e == cudaSuccess && serial) e = cudaStreamWaitEvent(b->master, prev, 0);
  const cudaError_t e2 = cudaStreamEndCapture(b->master, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess || st != EWH_OK) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (st != EWH_OK) return bfail(b, st, "batch member failed during capture: " + b->p[members.empty() ? 0 : members[0]]->err);
    return bfail(b, EWH_ECUDA, std::string("batch capture failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return bfail(b, EWH_ECUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(e));
  return EWH_OK;
}

// Order the members' own streams (residual replacements, mask uploads of the
// host decisions) before the next batch graph launch on the master stream.
bool members_before_master(ewh_batch* b, const std::vector<int>& members) {
  for (int k : members)
    if (cudaEventRecord(b->joins[k], b->p[k]->st) != cudaSuccess ||
        cudaStreamWaitEvent(b->master, b->joins[k], 0) != cudaSuccess)
      return false;
  return true;
}

// The batch's device-controlled CG windows: per member a while-conditional
// node whose body is one iteration of that member (its leapfrog launches, the
// Krylov kernels, the control kernel); the members' nodes run concurrently,
// or one after another when a member runs the resident solve.  Returns false
// (and the host polls every iteration) when the driver does not take it.
template <typename T>
bool build_batch_loop(ewh_batch* b, const std::vector<int>& members) {
  if (b->loop_graph) cudaGraphExecDestroy(b->loop_graph);
  b->loop_graph = nullptr;
  bool serial = false;
  if (sizeof(T) == 4)
    for (int k : members) serial = serial || is_resident_variant(b->p[k]->w32.variant);
  cudaGraph_t graph = nullptr;
  bool ok = cudaGraphCreate(&graph, 0) == cudaSuccess;
  b->loop_kernels.assign(b->p.size(), 0);
  cudaGraphNode_t prev = nullptr;
  for (int k : members) {
    if (!ok) break;
    ewh_ctx* ctx = b->p[k];
    if (ctx->implicit) {
      ok = false;
      break;
    }
    cudaGraphConditionalHandle h;
    ok = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    ok = ok && cudaGraphAddNode(&node, graph, (serial && prev) ? &prev : nullptr, nullptr, (serial && prev) ? 1 : 0,
                                &np) == cudaSuccess;
    if (!ok) break;
    ok = cudaStreamBeginCaptureToGraph(ctx->st, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                       cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (!ok) break;
    const long long l0 = ctx->launches;
    ok = cg_enqueue_iteration<T>(ctx, ctx->kx, ctx->kr, true, false) == EWH_OK &&
         launch_cg_control(h, ctx->g.nrhs, sc(ctx, S_RES), ctx->active, ctx->d_anchor, ctx->flags, ctx->d_loop,
                           ctx->d_hist, ctx->st) == cudaSuccess;
    b->loop_kernels[k] = ctx->launches - l0 + 1;
    ctx->launches = l0;  // captured, not run
    cudaGraph_t captured = nullptr;
    ok = cudaStreamEndCapture(ctx->st, &captured) == cudaSuccess && ok;
    prev = node;
  }
  ok = ok && cudaGraphInstantiate(&b->loop_graph, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  if (!ok) {
    if (b->loop_graph) cudaGraphExecDestroy(b->loop_graph);
    b->loop_graph = nullptr;
    cudaGetLastError();
    b->loop_failed = true;
    if (getenv("EWH_VERBOSE")) fprintf(stderr, "ewh: device-controlled batch CG unavailable: host polls each iteration\n");
    return false;
  }
  b->loop_members = members;
  return true;
}

template <typename T>
ewh_status batch_solve_T(ewh_batch* b, double tol, int maxit, double* const* v_out, ewh_solve_info* infos) {
  const int P = (int)b->p.size();
  std::vector<CgState> cs(P);
  std::vector<ewh_solve_info> inf(P);
  std::vector<ewh_status> status(P, EWH_OK);
  std::vector<int> fallback(P, 0);
  const double drop = sizeof(T) == 4 ? 0.1 : 0.0;
  const auto t0 = std::chrono::steady_clock::now();
  // right-hand sides b = Pi 0 (FP64) and the initial residuals, per member
  for (int k = 0; k < P; ++k) {
    ewh_ctx* ctx = b->p[k];
    ctx->history.clear();
    const long long n = total_unknowns(ctx);
    ewh_status s = run_wave<double>(ctx, nullptr, true);
    if (s != EWH_OK) return bfail(b, s, ctx->err);
    if (launch_unpack<double>(ctx->g, ctx->w64.acc, ctx->kb, nullptr, ctx->st) != cudaSuccess)
      return bfail(b, EWH_ECUDA, "unpack failed");
    ctx->launches += 1;
    inf[k].s_applies_fp64 += 1;
    s = mdot_dev(ctx, ctx->kb, ctx->kb, sc(ctx, S_BB));
    if (s != EWH_OK) return bfail(b, s, ctx->err);
    cudaMemsetAsync(ctx->kx, 0, sizeof(double) * n, ctx->st);
    cudaMemcpyAsync(ctx->kr, ctx->kb, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->st);
    s = cg_begin<T>(ctx, ctx->kr, tol, drop, cs[k]);
    if (s != EWH_OK) return bfail(b, s, ctx->err);
  }
  std::vector<int> members;
  for (int k = 0; k < P; ++k)
    if (cs[k].any_active) members.push_back(k);
  const int window = cg_window();
  while (!members.empty()) {
    bool dev = window > 1 && !b->loop_failed;
    if (dev && (members != b->loop_members || !b->loop_graph)) dev = build_batch_loop<T>(b, members);
    if (dev) {
      // a window of iterations of every member under device control; then, per
      // member, the host decisions of its window's last iteration
      for (int k : members) {
        ewh_ctx* ctx = b->p[k];
        const int R = ctx->g.nrhs;
        for (int q = 0; q < R; ++q) ctx->h_anchor[q] = cs[k].anchor[q];
        ctx->h_anchor[R] = tol;
        ctx->h_anchor[R + 1] = drop;
        ctx->h_loop[0] = 0;
        ctx->h_loop[1] = std::max(1, std::min(window, maxit - inf[k].iters));
        if (cudaMemcpyAsync(ctx->d_anchor, ctx->h_anchor, sizeof(double) * (R + 2), cudaMemcpyHostToDevice,
                            b->master) != cudaSuccess ||
            cudaMemcpyAsync(ctx->d_loop, ctx->h_loop, sizeof(int) * 2, cudaMemcpyHostToDevice, b->master) !=
                cudaSuccess)
          return bfail(b, EWH_ECUDA, "batch window setup failed");
      }
      bool ok = members_before_master(b, members) && cudaGraphLaunch(b->loop_graph, b->master) == cudaSuccess;
      for (int k : members) {
        ewh_ctx* ctx = b->p[k];
        const int R = ctx->g.nrhs;
        ok = ok &&
             cudaMemcpyAsync(ctx->h_scal, ctx->scal, sizeof(double) * S_N * R, cudaMemcpyDeviceToHost, b->master) ==
                 cudaSuccess &&
             cudaMemcpyAsync(ctx->h_act, ctx->active, sizeof(int) * R, cudaMemcpyDeviceToHost, b->master) ==
                 cudaSuccess &&
             cudaMemcpyAsync(ctx->h_flag, ctx->flags, sizeof(int), cudaMemcpyDeviceToHost, b->master) == cudaSuccess &&
             cudaMemcpyAsync(ctx->h_loop, ctx->d_loop, sizeof(int) * 2, cudaMemcpyDeviceToHost, b->master) ==
                 cudaSuccess &&
             cudaMemcpyAsync(ctx->h_hist, ctx->d_hist, sizeof(double) * window, cudaMemcpyDeviceToHost, b->master) ==
                 cudaSuccess;
      }
      if (!ok || cudaStreamSynchronize(b->master) != cudaSuccess)
        return bfail(b, EWH_ECUDA, std::string("batch window failed: ") + cudaGetErrorString(cudaGetLastError()));
      std::vector<int> next;
      for (int k : members) {
        ewh_ctx* ctx = b->p[k];
        const int it = ctx->h_loop[0];
        if (it < 1) return bfail(b, EWH_ECUDA, "device-controlled batch window ran no iteration");
        b->launches += (long long)it * b->loop_kernels[k];
        ctx->loop_steps[sizeof(T) == 4 ? 1 : 0] += (long long)it * ctx->nt * ctx->periods;
        ctx->loop_waves[sizeof(T) == 4 ? 1 : 0] += it;
        for (int i = 0; i + 1 < it; ++i) {  // iterations that needed no host decision
          ctx->history.push_back(ctx->h_hist[i]);
          ++inf[k].iters;
          if (sizeof(T) == 8) ++inf[k].s_applies_fp64;
          else ++inf[k].s_applies;
        }
        ewh_status s = cg_after_iteration<T>(ctx, ctx->kx, ctx->kr, cs[k], &inf[k]);
        if (s == EWH_EBREAKDOWN) {
          fallback[k] = 1;
          continue;
        }
        if (s != EWH_OK) return bfail(b, s, ctx->err);
        if (cs[k].any_active && inf[k].iters < maxit) next.push_back(k);
      }
      members.swap(next);
      continue;
    }
    if (members != b->graph_members || !b->iter_graph) {
      if (b->iter_graph) cudaGraphExecDestroy(b->iter_graph);
      b->iter_graph = nullptr;
      ewh_status s = capture_branches(
          b, members, [&](int k) { return cg_enqueue_iteration<T>(b->p[k], b->p[k]->kx, b->p[k]->kr, true); },
          &b->iter_graph);
      if (s != EWH_OK) return s;
      b->graph_members = members;
    }
    if (!members_before_master(b, members) || cudaGraphLaunch(b->iter_graph, b->master) != cudaSuccess ||
        cudaStreamSynchronize(b->master) != cudaSuccess)
      return bfail(b, EWH_ECUDA, std::string("batch iteration failed: ") + cudaGetErrorString(cudaGetLastError()));
    std::vector<int> next;
    for (int k : members) {
      ewh_ctx* ctx = b->p[k];
      ctx->launches += 0;  // counted when captured below
      ewh_status s = cg_after_iteration<T>(ctx, ctx->kx, ctx->kr, cs[k], &inf[k]);
      if (s == EWH_EBREAKDOWN) {
        fallback[k] = 1;
        continue;
      }
      if (s != EWH_OK) return bfail(b, s, ctx->err);
      if (cs[k].any_active && inf[k].iters < maxit) next.push_back(k);
    }
    // launches of one batched iteration: per member 1 pack + steps + 5 Krylov kernels
    for (int k : members) {
      const Wave<T>& w = wave_of<T>(b->p[k]);
      b->launches += 6 + (w.graph_S_kernels ? w.graph_S_kernels : 0);
    }
    members.swap(next);
  }
  // members whose FP32 operator lost definiteness continue alone in FP64;
  // members whose FP64 CG broke down continue with MINRES (as ewh_solve)
  for (int k = 0; k < P; ++k) {
    ewh_ctx* ctx = b->p[k];
    double rel = cg_worst_true(cs[k]);
    if (fallback[k]) {
      if (sizeof(T) == 4) {
        ewh_status s = true_residual(ctx, ctx->kx, ctx->kr, &rel);
        if (s != EWH_OK) return bfail(b, s, ctx->err);
        ++inf[k].s_applies_fp64;
        ctx->err = "no error";
        status[k] = run_cg<double>(ctx, ctx->kx, ctx->kr, tol, maxit, 0.0, &inf[k], &rel);
      } else {
        status[k] = EWH_EBREAKDOWN;
      }
      if (status[k] == EWH_EBREAKDOWN) {
        ewh_status s = minres_after_breakdown(ctx, tol, maxit, &inf[k], &rel, &status[k]);
        if (s != EWH_OK) return bfail(b, s, ctx->err);
      }
    }
    inf[k].rel_res = rel;
    if (status[k] == EWH_OK && !(rel <= tol)) {
      status[k] = EWH_ENOTCONV;
      ctx->err = "not converged: relative residual " + std::to_string(rel) + " > tol";
    }
    const long long n = total_unknowns(ctx);
    if (v_out && v_out[k] &&
        (cudaMemcpyAsync(v_out[k], ctx->kx, sizeof(double) * n, cudaMemcpyDefault, ctx->st) != cudaSuccess ||
         cudaStreamSynchronize(ctx->st) != cudaSuccess))
      return bfail(b, EWH_ECUDA, "copy of a batch solution failed");
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  ewh_status first = EWH_OK;
  for (int k = 0; k < P; ++k) {
    inf[k].seconds = secs;
    inf[k].status = status[k];
    if (infos) infos[k] = inf[k];
    if (first == EWH_OK && status[k] != EWH_OK) {
      first = status[k];
      b->err = "member " + std::to_string(k) + ": " + b->p[k]->err;
    }
  }
  return first;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
namespace {

// Context creation; xmap/ymap (node coordinates of a mapped 2D grid) may be null.
ewh_status create_impl(const ewh_grid_desc* desc, const double* xmap, const double* ymap, const double* rho,
                       const double* lambda, const double* mu, double omega, const double* forcing, int nrhs,
                       void* cuda_stream, ewh_ctx** out) {
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
  const bool mapped = xmap != nullptr;
  std::vector<double> hmet;  // mapped grids: (y_r, -x_r, -y_q, x_q, 1/J, J) per node
  double* d_met = nullptr;
  if (mapped) {  // Section 4.1, curvilinear form: metric terms from the SBP derivative of the mapping
    if (dim != 2 || desc->order != 4)
      return fail(nullptr, EWH_EINVAL, "mapped grids need dim 2 and order 4");
    std::vector<double> hx(full), hy(full);
    if (fetch(xmap, hx) != cudaSuccess || fetch(ymap, hy) != cudaSuccess) {
      cudaGetLastError();
      return fail(nullptr, EWH_EINVAL, "cannot read the node coordinates");
    }
    for (long long i = 0; i < full; ++i)
      if (!std::isfinite(hx[i]) || !std::isfinite(hy[i]))
        return fail(nullptr, EWH_EINVAL, "node coordinates must be finite");
    hmet.resize(6 * full);
    double *d_xy = nullptr;
    cudaStream_t ts = nullptr;
    bool ok = cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) == cudaSuccess &&
              cudaMalloc(&d_xy, sizeof(double) * 2 * full) == cudaSuccess &&
              cudaMalloc(&d_met, sizeof(double) * 6 * full) == cudaSuccess &&
              cudaMemcpyAsync(d_xy, hx.data(), sizeof(double) * full, cudaMemcpyHostToDevice, ts) == cudaSuccess &&
              cudaMemcpyAsync(d_xy + full, hy.data(), sizeof(double) * full, cudaMemcpyHostToDevice, ts) == cudaSuccess &&
              launch_curv_metrics(desc->n[0], desc->n[1], desc->h, d_xy, d_xy + full, d_met, ts) == cudaSuccess &&
              cudaMemcpyAsync(hmet.data(), d_met, sizeof(double) * 6 * full, cudaMemcpyDeviceToHost, ts) == cudaSuccess &&
              cudaStreamSynchronize(ts) == cudaSuccess;
    cudaFree(d_xy);
    if (ts) cudaStreamDestroy(ts);
    if (!ok) {
      cudaGetLastError();
      cudaFree(d_met);
      return fail(nullptr, EWH_ECUDA, "metric computation failed (no CUDA device?)");
    }
    for (long long i = 0; i < full; ++i)
      if (!(hmet[5 * full + i] > 0.0) || !std::isfinite(hmet[5 * full + i])) {
        cudaFree(d_met);
        return fail(nullptr, EWH_EINVAL, "mapping not orientation preserving at node " + std::to_string(i) + " (J <= 0)");
      }
  }
  double speed2 = 0.0;
  for (long long i = 0; i < full; ++i) {
    const double r = hr[i], l = hl[i], m = hm[i];
    if (!std::isfinite(r) || !std::isfinite(l) || !std::isfinite(m) || !(r > 0.0) || !(m > 0.0) ||
        !(l > -2.0 * m / dim)) {
      cudaFree(d_met);
      return fail(nullptr, EWH_EINVAL,
                  "invalid medium at node " + std::to_string(i) + ": need finite rho > 0, mu > 0, lambda > -2 mu / dim");
    }
    double c2 = (l + (dim + 1) * m) / r;
    if (mapped) {  // (|grad q|^2 + |grad r|^2) / 2 scales the Cartesian bound
      const double a0 = hmet[i], a1 = hmet[full + i], a2 = hmet[2 * full + i], a3 = hmet[3 * full + i];
      const double iJ = hmet[4 * full + i];
      c2 *= 0.5 * (a0 * a0 + a1 * a1 + a2 * a2 + a3 * a3) * iJ * iJ;
    }
    if (c2 > speed2) speed2 = c2;
  }
  std::vector<double> hf;  // mapped grids: J f, so that (J f) / (rho J) = f / rho
  if (mapped) {
    for (long long i = 0; i < full; ++i) {
      hr[i] *= hmet[5 * full + i];  // the mass density rho J
      hl[i] *= hmet[4 * full + i];  // lambda / J and mu / J: the stress kernels take
      hm[i] *= hmet[4 * full + i];  // J times the physical gradient
    }
    if (forcing) {
      hf.resize((size_t)full * dim * nrhs);
      cudaPointerAttributes at;
      if (cudaPointerGetAttributes(&at, forcing) == cudaSuccess &&
          (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)) {
        if (cudaMemcpy(hf.data(), forcing, sizeof(double) * hf.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
          cudaGetLastError();
          cudaFree(d_met);
          return fail(nullptr, EWH_EINVAL, "cannot read the forcing");
        }
      } else {
        cudaGetLastError();
        std::memcpy(hf.data(), forcing, sizeof(double) * hf.size());
      }
      for (size_t k = 0; k < hf.size(); ++k) hf[k] *= hmet[5 * full + (long long)(k % full)];
      forcing = hf.data();
    }
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
  g.mapped = mapped ? 1 : 0;
  for (int a = 0; a < 3; ++a) {
    g.n[a] = a < dim ? desc->n[a] : 1;
    g.lo_free[a] = a < dim ? (desc->bc[2 * a] == EWH_BC_FREE) : 1;
    g.hi_free[a] = a < dim ? (desc->bc[2 * a + 1] == EWH_BC_FREE) : 1;
  }
  for (int a = 0; a < 3; ++a) {
    if (a < dim) {
      const int rounded = ((g.n[a] + TILE_ROUND - 1) / TILE_ROUND) * TILE_ROUND;
      g.np[a] = rounded + (a == 0 ? PAD3X : 2 * PAD);
      g.off[a] = g.lo_free[a] ? 0 : 1;
      g.nu[a] = g.n[a] - (g.lo_free[a] ? 0 : 1) - (g.hi_free[a] ? 0 : 1);
    } else {
      g.np[a] = 1;
      g.off[a] = 0;
      g.nu[a] = 1;
    }
  }
  g.pz = dim == 3 ? PAD : 0;
  g.padx = 8 - g.off[0];
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
      cudaFree(d_met);
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
  if (desc->implicit) {  // Section 4.4: alpha (eq. alpha), or 2 for the unmodified scheme
    const double wd = omega * ctx->dt;
    ctx->implicit = 1;
    ctx->alpha = ctx->corrected ? std::cos(wd) * (2.0 + wd * wd) : 2.0;
    ctx->omega_t = std::cos(wd) > 0.0 ? 2.0 * std::sin(wd / 2.0) / (ctx->dt * std::sqrt(std::cos(wd))) : NAN;
    ctx->kt = 0.0;
    if (!(std::fabs(ctx->alpha) < 2.0) && ctx->corrected) {
      cudaFree(d_met);
      delete ctx;
      return fail(nullptr, EWH_EINVAL, "implicit scheme unstable: |alpha| >= 2 (use nt >= 5)");
    }
  }

  // CUDA resources
  auto bail = [&](ewh_status s, const std::string& m) {
    g_create_error = m;
    cudaFree(d_met);
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

  ewh_status s = build_wave<double>(ctx, ctx->w64, d_r, d_l, d_m, d_f, d_met);
  if (s == EWH_OK && ctx->precision == EWH_FP32_STENCIL)
    s = build_wave<float>(ctx, ctx->w32, d_r, d_l, d_m, d_f, d_met);
  const long long n = total_unknowns(ctx);
  ctx->nblk = dot_blocks(g);
  if (s == EWH_OK) {
    ok = alloc_zero(&ctx->kx, n, ctx->st) == cudaSuccess && alloc_zero(&ctx->kr, n, ctx->st) == cudaSuccess &&
         alloc_zero(&ctx->kp, n, ctx->st) == cudaSuccess && alloc_zero(&ctx->kq, n, ctx->st) == cudaSuccess &&
         alloc_zero(&ctx->kb, n, ctx->st) == cudaSuccess && alloc_zero(&ctx->kd, n, ctx->st) == cudaSuccess &&
         alloc_zero(&ctx->ktmp, n, ctx->st) == cudaSuccess && alloc_zero(&ctx->mw, g.nodes, ctx->st) == cudaSuccess &&
         alloc_zero(&ctx->kar, n, ctx->st) == cudaSuccess && alloc_zero(&ctx->kap, n, ctx->st) == cudaSuccess &&
         alloc_zero(&ctx->part, (size_t)ctx->nblk * nrhs, ctx->st) == cudaSuccess &&
         alloc_zero(&ctx->scal, (size_t)S_N * nrhs, ctx->st) == cudaSuccess &&
         alloc_zero(&ctx->active, nrhs, ctx->st) == cudaSuccess && alloc_zero(&ctx->flags, 1, ctx->st) == cudaSuccess &&
         cudaMallocHost(&ctx->h_scal, sizeof(double) * S_N * nrhs) == cudaSuccess &&
         cudaMallocHost(&ctx->h_act, sizeof(int) * nrhs) == cudaSuccess &&
         cudaMallocHost(&ctx->h_flag, sizeof(int)) == cudaSuccess &&
         alloc_zero(&ctx->d_anchor, nrhs + 2, ctx->st) == cudaSuccess &&
         alloc_zero(&ctx->d_loop, 2, ctx->st) == cudaSuccess &&
         alloc_zero(&ctx->d_hist, CG_WINDOW_MAX, ctx->st) == cudaSuccess &&
         cudaMallocHost(&ctx->h_anchor, sizeof(double) * (nrhs + 2)) == cudaSuccess &&
         cudaMallocHost(&ctx->h_loop, sizeof(int) * 2) == cudaSuccess &&
         cudaMallocHost(&ctx->h_hist, sizeof(double) * CG_WINDOW_MAX) == cudaSuccess;
    if (ok && ctx->implicit) {
      for (double** q : {&ctx->iu_prev, &ctx->iu, &ctx->iu_next, &ctx->ig, &ctx->ir, &ctx->ip, &ctx->iq, &ctx->iacc})
        ok = ok && alloc_zero(q, n, ctx->st) == cudaSuccess;
      ok = ok && alloc_zero(&ctx->iscal, (size_t)I_N * nrhs, ctx->st) == cudaSuccess;
      if (ok && forcing) ok = alloc_zero(&ctx->ifr, n, ctx->st) == cudaSuccess;
    }
    if (!ok) {
      cudaGetLastError();
      s = fail(ctx, EWH_ENOMEM, "device allocation of the Krylov workspace failed");
    }
  }
  if (s == EWH_OK && ctx->ifr) {  // f / rho at the unknowns, dense (from the padded FP64 field)
    if (launch_unpack<double>(g, ctx->w64.frho, ctx->ifr, nullptr, ctx->st) != cudaSuccess)
      s = fail(ctx, EWH_ECUDA, "forcing unpack failed");
    ctx->launches += 1;
  }
  if (s == EWH_OK) {
    if (launch_fill_mass(g, ctx->order, d_r, desc->h, ctx->mw, ctx->st) != cudaSuccess)
      s = fail(ctx, EWH_ECUDA, "mass kernel launch failed");
    ctx->launches += 1;
  }
  cudaError_t e = cudaStreamSynchronize(ctx->st);
  cudaFree(d_met);
  d_met = nullptr;
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

}  // namespace

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
  cudaFree(ctx->kar);
  cudaFree(ctx->kap);
  for (double* q : {ctx->iu_prev, ctx->iu, ctx->iu_next, ctx->ig, ctx->ir, ctx->ip, ctx->iq, ctx->iacc, ctx->ifr,
                    ctx->iscal})
    cudaFree(q);
  cudaFree(ctx->mw);
  cudaFree(ctx->part);
  cudaFree(ctx->scal);
  cudaFree(ctx->active);
  cudaFree(ctx->flags);
  if (ctx->h_scal) cudaFreeHost(ctx->h_scal);
  if (ctx->h_act) cudaFreeHost(ctx->h_act);
  if (ctx->h_flag) cudaFreeHost(ctx->h_flag);
  cudaFree(ctx->d_anchor);
  cudaFree(ctx->d_loop);
  cudaFree(ctx->d_hist);
  if (ctx->h_anchor) cudaFreeHost(ctx->h_anchor);
  if (ctx->h_loop) cudaFreeHost(ctx->h_loop);
  if (ctx->h_hist) cudaFreeHost(ctx->h_hist);
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
  return create_impl(desc, nullptr, nullptr, rho, lambda, mu, omega, forcing, nrhs, cuda_stream, out);
}

ewh_status ewh_create_mapped(const ewh_grid_desc* desc, const double* x, const double* y, const double* rho,
                             const double* lambda, const double* mu, double omega, const double* forcing, int nrhs,
                             void* cuda_stream, ewh_ctx** out) {
  if (out) *out = nullptr;
  if (!x || !y) return fail(nullptr, EWH_EINVAL, "x and y (node coordinates) are required");
  return create_impl(desc, x, y, rho, lambda, mu, omega, forcing, nrhs, cuda_stream, out);
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
  info->kernel_variant[0] = ctx->w64.variant;
  info->kernel_variant[1] = ctx->w32.variant;
  for (int k = 0; k < 10; ++k) info->resident[k] = -1;
  const int v = ctx->w32.variant;
  if (is_resident_variant(v)) {
    const ResidentPlan& p = ctx->w32.rplan[v - VARIANT_RESIDENT];
    const int r[10] = {p.shape, p.px, p.py, p.bx, p.ex, p.by, RS_SHAPE_THREADS[p.shape], RS_SHAPE_PAIRS[p.shape],
                       p.rg, p.groups};
    for (int k = 0; k < 10; ++k) info->resident[k] = r[k];
  }
  return EWH_OK;
}

ewh_status ewh_set_grid_wait(ewh_ctx* ctx, long long ns) {
  if (!ctx) return EWH_EINVAL;
  if (ns < 0) return fail(ctx, EWH_EINVAL, "grid wait limit must be >= 0 ns");
  if (!ctx->w32.bar) return EWH_OK;  // this context never runs the on-chip solve
  const unsigned long long v = (unsigned long long)ns;
  if (cudaStreamSynchronize(ctx->st) != cudaSuccess ||
      cudaMemcpy(ctx->w32.bar + 2, &v, sizeof(v), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(ctx, EWH_ECUDA, "setting the grid wait limit failed");
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
  if (ctx->implicit) {
    s = implicit_wave(ctx, nullptr, true);
    if (s == EWH_OK && cudaMemcpyAsync(b_out, ctx->iacc, sizeof(double) * total_unknowns(ctx),
                                       cudaMemcpyDeviceToDevice, ctx->st) != cudaSuccess)
      s = fail(ctx, EWH_ECUDA, "copy failed");
  } else if (ctx->precision == EWH_FP64) {
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
                           &ctx->launches, w.met) != cudaSuccess ||
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

ewh_status ewh_solve_cr(ewh_ctx* ctx, double tol, int maxit, const double* x0_or_null, double* v_out,
                        ewh_solve_info* info) {
  if (!ctx || !v_out) return fail(ctx, EWH_EINVAL, "null argument");
  if (!(tol > 0.0) || maxit < 0) return fail(ctx, EWH_EINVAL, "tol must be > 0 and maxit >= 0");
  if (!ctx->has_forcing) return fail(ctx, EWH_EINVAL, "problem was created without forcing");
  ewh_status s = check_async(ctx);
  if (s != EWH_OK) return s;
  const auto t0 = std::chrono::steady_clock::now();
  enter(ctx);
  ewh_solve_info inf{};
  s = solve_impl(ctx, tol, maxit, x0_or_null, v_out, &inf, 1);
  leave(ctx);
  cudaStreamSynchronize(ctx->st);
  inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  inf.status = s;
  if (info) *info = inf;
  if (s == EWH_OK) s = check_async(ctx);
  return s;
}

ewh_status ewh_solve_minres(ewh_ctx* ctx, double tol, int maxit, const double* x0_or_null, double* v_out,
                            ewh_solve_info* info) {
  if (!ctx || !v_out) return fail(ctx, EWH_EINVAL, "null argument");
  if (!(tol > 0.0) || maxit < 0) return fail(ctx, EWH_EINVAL, "tol must be > 0 and maxit >= 0");
  if (!ctx->has_forcing) return fail(ctx, EWH_EINVAL, "problem was created without forcing");
  ewh_status s = check_async(ctx);
  if (s != EWH_OK) return s;
  const auto t0 = std::chrono::steady_clock::now();
  enter(ctx);
  ewh_solve_info inf{};
  s = solve_impl(ctx, tol, maxit, x0_or_null, v_out, &inf, 2);
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

void ewh_batch_destroy(ewh_batch* b) {
  if (!b) return;
  if (b->master) cudaStreamSynchronize(b->master);
  if (b->iter_graph) cudaGraphExecDestroy(b->iter_graph);
  if (b->loop_graph) cudaGraphExecDestroy(b->loop_graph);
  for (auto c : b->p) ewh_destroy(c);
  for (auto e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->master) cudaStreamDestroy(b->master);
  delete b;
}

ewh_status ewh_batch_create(const ewh_problem* probs, int nprob, void* cuda_stream, ewh_batch** out) {
  if (!out) return fail(nullptr, EWH_EINVAL, "out is NULL");
  *out = nullptr;
  if (!probs || nprob < 1 || nprob > 4096) return fail(nullptr, EWH_EINVAL, "nprob must be in [1, 4096]");
  for (int k = 1; k < nprob; ++k)
    if (probs[k].desc.dim != probs[0].desc.dim || probs[k].desc.order != probs[0].desc.order ||
        probs[k].desc.precision != probs[0].desc.precision)
      return fail(nullptr, EWH_EINVAL, "batch members must share dim, order and precision");
  ewh_batch* b = new ewh_batch();
  b->user_stream = (cudaStream_t)cuda_stream;
  b->precision = probs[0].desc.precision;
  for (int k = 0; k < nprob; ++k)
    if (probs[k].desc.implicit) return fail(nullptr, EWH_EINVAL, "batch members must use the explicit scheme");
  for (int k = 0; k < nprob; ++k) {
    ewh_ctx* c = nullptr;
    ewh_status s = ewh_create(&probs[k].desc, probs[k].rho, probs[k].lambda, probs[k].mu, probs[k].omega,
                              probs[k].forcing, probs[k].nrhs, cuda_stream, &c);
    if (s != EWH_OK) {
      const std::string m = "member " + std::to_string(k) + ": " + g_create_error;
      ewh_batch_destroy(b);
      g_create_error = m;
      return s;
    }
    c->batch_member = true;
    b->p.push_back(c);
  }
  b->joins.resize(nprob, nullptr);
  bool ok = cudaStreamCreateWithFlags(&b->master, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; ok && k < nprob; ++k)
    ok = cudaEventCreateWithFlags(&b->joins[k], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    ewh_batch_destroy(b);
    return fail(nullptr, EWH_ECUDA, "cannot create batch streams/events");
  }
  *out = b;
  return EWH_OK;
}

ewh_status ewh_batch_member(ewh_batch* b, int k, ewh_ctx** ctx) {
  if (!b || !ctx || k < 0 || k >= (int)b->p.size()) return EWH_EINVAL;
  *ctx = b->p[k];
  return EWH_OK;
}

long long ewh_batch_kernel_launches(const ewh_batch* b) {
  if (!b) return 0;
  long long n = b->launches;
  for (auto c : b->p) n += c->launches;
  return n;
}

const char* ewh_batch_last_error(const ewh_batch* b) { return b ? b->err.c_str() : g_create_error.c_str(); }

ewh_status ewh_batch_apply_S(ewh_batch* b, const double* const* v_in, double* const* v_out) {
  if (!b || !v_in || !v_out) return EWH_EINVAL;
  std::vector<int> members;
  for (int k = 0; k < (int)b->p.size(); ++k) {
    members.push_back(k);
    const ewh_status s0 = b->precision == EWH_FP64 ? ensure_graph<double>(b->p[k], false)
                                                   : ensure_graph<float>(b->p[k], false);
    if (s0 != EWH_OK) return bfail(b, s0, b->p[k]->err);
  }
  cudaEventRecord(b->fork, b->user_stream);
  cudaStreamWaitEvent(b->master, b->fork, 0);
  cudaGraphExec_t ge = nullptr;
  auto body = [&](int k) -> ewh_status {
    ewh_ctx* ctx = b->p[k];
    if (b->precision == EWH_FP64) {
      Wave<double>& w = ctx->w64;
      if (launch_pack<double>(ctx->g, v_in[k], w.u_a, ctx->st) != cudaSuccess) return EWH_ECUDA;
      long long cnt = 0;
      if (enqueue_steps<double>(ctx, w, false, &cnt) != cudaSuccess) return EWH_ECUDA;
      if (launch_unpack<double>(ctx->g, w.acc, v_out[k], nullptr, ctx->st) != cudaSuccess) return EWH_ECUDA;
      b->launches += cnt + 2;
    } else {
      Wave<float>& w = ctx->w32;
      if (launch_pack<float>(ctx->g, v_in[k], w.u_a, ctx->st) != cudaSuccess) return EWH_ECUDA;
      long long cnt = 0;
      if (enqueue_steps<float>(ctx, w, false, &cnt) != cudaSuccess) return EWH_ECUDA;
      if (launch_unpack<float>(ctx->g, w.acc, v_out[k], nullptr, ctx->st) != cudaSuccess) return EWH_ECUDA;
      b->launches += cnt + 2;
    }
    return EWH_OK;
  };
  ewh_status s = capture_branches(b, members, body, &ge);
  if (s != EWH_OK) return s;
  cudaError_t e = cudaGraphLaunch(ge, b->master);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->master);
  cudaGraphExecDestroy(ge);
  if (e != cudaSuccess) return bfail(b, EWH_ECUDA, std::string("batch apply failed: ") + cudaGetErrorString(e));
  cudaEventRecord(b->fork, b->master);
  cudaStreamWaitEvent(b->user_stream, b->fork, 0);
  return EWH_OK;
}

ewh_status ewh_batch_solve(ewh_batch* b, double tol, int maxit, double* const* v_out, ewh_solve_info* infos) {
  if (!b) return EWH_EINVAL;
  if (!(tol > 0.0) || maxit < 0) return bfail(b, EWH_EINVAL, "tol must be > 0 and maxit >= 0");
  for (auto c : b->p)
    if (!c->has_forcing) return bfail(b, EWH_EINVAL, "every member needs forcing to be solved");
  cudaEventRecord(b->fork, b->user_stream);
  for (auto c : b->p) cudaStreamWaitEvent(c->st, b->fork, 0);
  ewh_status s = b->precision == EWH_FP64 ? batch_solve_T<double>(b, tol, maxit, v_out, infos)
                                          : batch_solve_T<float>(b, tol, maxit, v_out, infos);
  for (auto c : b->p) {
    cudaEventRecord(c->ev_out, c->st);
    cudaStreamWaitEvent(b->user_stream, c->ev_out, 0);
  }
  return s;
}

ewh_status ewh_get_stats(ewh_ctx* ctx, ewh_stats* out) {
  if (!ctx || !out) return EWH_EINVAL;
  if (cudaStreamSynchronize(ctx->st) != cudaSuccess) return fail(ctx, EWH_ECUDA, "synchronise failed");
  collect_timing(ctx);
  for (int k = 0; k < 2; ++k) {
    out->wave_ms[k] = ctx->wave_ms[k];
    out->steps[k] = ctx->wave_steps[k];
    out->waves[k] = ctx->wave_count[k];
    out->loop_steps[k] = ctx->loop_steps[k];
    out->loop_waves[k] = ctx->loop_waves[k];
  }
  out->launches = ctx->launches;
  out->grid_wait_timeouts = 0;
  if (ctx->w32.bar) {
    unsigned n = 0;
    if (cudaMemcpy(&n, ctx->w32.bar + 4, sizeof(n), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(ctx, EWH_ECUDA, "reading the grid wait counter failed");
    out->grid_wait_timeouts = (long long)n - ctx->grid_timeouts_base;
  }
  return EWH_OK;
}

ewh_status ewh_reset_stats(ewh_ctx* ctx) {
  if (!ctx) return EWH_EINVAL;
  if (cudaStreamSynchronize(ctx->st) != cudaSuccess) return fail(ctx, EWH_ECUDA, "synchronise failed");
  collect_timing(ctx);
  for (int k = 0; k < 2; ++k)
    ctx->wave_ms[k] = 0, ctx->wave_steps[k] = 0, ctx->wave_count[k] = 0, ctx->loop_steps[k] = 0,
    ctx->loop_waves[k] = 0;
  ctx->launches = 0;
  if (ctx->w32.bar) {
    unsigned n = 0;
    if (cudaMemcpy(&n, ctx->w32.bar + 4, sizeof(n), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(ctx, EWH_ECUDA, "reading the grid wait counter failed");
    ctx->grid_timeouts_base = (long long)n;
  }
  return EWH_OK;
}

}  // extern "C"
