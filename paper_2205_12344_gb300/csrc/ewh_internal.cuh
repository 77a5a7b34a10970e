// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace ewh {

// Padding (ghost layers, always zero) around the full node grid of every
// device field.  Order 4 reads up to 6 nodes beyond a tile; tiles are at most
// 32 wide and the padded extents are rounded up to a multiple of 32 first.
// Along x the fields pad 7 or 8 nodes before and at least 8 after the grid
// (see Geom::padx), with np[0] = rounded + PAD3X.
constexpr int PAD = 6;
constexpr int TILE_ROUND = 32;
constexpr int PAD3X = 16;

// Geometry of one problem in the padded device layout.
struct Geom {
  int dim;
  int n[3];        // full-grid nodes per axis (n[2] = 1 in 2D)
  int lo_free[3];  // 1 if the low side of the axis is a free surface
  int hi_free[3];
  int np[3];       // padded extents (np[2] = 1 in 2D)
  int padx;        // padding before x = 0: 8 - off[0], so the first unknown node of every row
                   // sits at a padded x that is a multiple of 4 (16-byte aligned rows of unknown
                   // pairs for vector and bulk-tensor access)
  int pz;          // padding along z (PAD in 3D, 0 in 2D)
  long long plane; // np[0] * np[1]
  long long field; // elements of one padded component: plane * np[2]
  int nu[3];       // unknown nodes per axis
  int off[3];      // full-grid index of the first unknown node per axis
  long long nodes; // unknown nodes per component
  int nrhs;
  int variant;     // step-kernel variant chosen by the autotuner (host side)
  int mapped;      // 1: curvilinear 2D grid (order 4): fluxes through WaveFields::met
};

// Boundary closure of the diagonal-norm 2-4 summation-by-parts first
// derivative (rows 0..3 = the first four nodes of a line, columns 0..5); the
// last four rows are the negated mirror.  Norm weight of the boundary row:
// 17/48.
constexpr double SBP_CLOSURE[4][6] = {{-24.0 / 17, 59.0 / 34, -4.0 / 17, -3.0 / 34, 0.0, 0.0},
                                      {-0.5, 0.0, 0.5, 0.0, 0.0, 0.0},
                                      {4.0 / 43, -59.0 / 86, 0.0, 59.0 / 86, -4.0 / 43, 0.0},
                                      {3.0 / 98, 0.0, -59.0 / 98, 0.0, 32.0 / 49, -4.0 / 49}};

// Number of step-kernel variants worth timing for a geometry/order.
inline int step_variant_count(int dim, int order) {
  if (dim == 2 && order == 4) return 5;  // split with 4 block shapes, fused
  if (dim == 2 && order == 2) return 3;  // tile heights 8, 4, 16
  if (dim == 3 && order == 4) return 3;  // stress + divergence pair, fused z-march 32x16 and 32x8 (FP32)
  return 1;
}

__host__ __device__ inline long long pidx(const Geom& g, int rhs, int comp, int x, int y, int z) {
  return ((long long)(rhs * g.dim + comp)) * g.field +
         (long long)(z + g.pz) * g.plane + (long long)(y + PAD) * g.np[0] + (x + g.padx);
}

// 1 if full-grid node (x, y, z) is an unknown.
__host__ __device__ inline bool is_unknown(const Geom& g, int x, int y, int z) {
  if (x < 0 || x >= g.n[0] || y < 0 || y >= g.n[1] || z < 0 || z >= g.n[2]) return false;
  if (x == 0 && !g.lo_free[0]) return false;
  if (x == g.n[0] - 1 && !g.hi_free[0]) return false;
  if (y == 0 && !g.lo_free[1]) return false;
  if (y == g.n[1] - 1 && !g.hi_free[1]) return false;
  if (g.dim == 3) {
    if (z == 0 && !g.lo_free[2]) return false;
    if (z == g.n[2] - 1 && !g.hi_free[2]) return false;
  }
  return true;
}

// Scalars of one time step (host-computed in FP64).
struct StepScalars {
  double kt;     // c dt^2
  double cosn;   // cos(w t_n) of the level whose operator is applied
  double w0;     // filter weight of u^0 (first step only)
  double wnew;   // filter weight of the new level
};

enum StepMode { STEP_FIRST = 0, STEP_MID = 1, STEP_LAST = 2 };

// Plan of the fused marching FP32 order-4 steps: bulk-tensor maps of both u
// buffers, the persistent grid and the control words (wait limit in ns at
// [2..3] as a u64, give-up count at [4]).
// 3D z-march (ewh_zmarch.cu), shapes k = 0 tiles of 32 x 16 nodes (one CTA
// per SM), k = 1 tiles of 32 x 8 (two CTAs per SM); 2D y-march
// (ewh_ymarch.cu), slot 0: strips of 60 columns, one warp per CTA.
constexpr int ZM_MAP_BYTES = 128;
constexpr int ZM_SHAPES = 2;
struct ZmPlan {
  int ok[ZM_SHAPES] = {0, 0};
  int grid[ZM_SHAPES] = {0, 0};
  int shx[ZM_SHAPES] = {0, 0};  // tile origins before the first unknown (x, y)
  int shy[ZM_SHAPES] = {0, 0};
  const float* u_a = nullptr;  // the buffers the maps describe
  const float* u_b = nullptr;
  unsigned* ctl = nullptr;
  alignas(64) unsigned char tmap[ZM_SHAPES][2][ZM_MAP_BYTES];
};

// Pointers of one wave solve (padded fields, all right-hand sides).
template <typename T>
struct WaveFields {
  T* u_cur;        // u^n (halo reads)
  T* u_next;       // u^{n+1}
  T* delta;        // u^{n+1} - u^n (in place)
  T* acc;          // trapezoid accumulator
  const T* lam;    // medium (shared by the right-hand sides)
  const T* mu;
  const T* irh2;   // 1 / (rho h^2)
  const T* frho;   // f / rho per rhs and component, or nullptr (S apply)
  T* sigma;        // order-4 stress scratch (dim*(dim+1)/2 fields per rhs) or nullptr
  const T* met = nullptr;  // mapped grids: 4 planes (y_r, -x_r, -y_q, x_q) of one padded component
  const ZmPlan* zm = nullptr;  // order 4, FP32: plan of the fused marching step (host pointer)
};

// ---- launchers (ewh_stencil.cu) -------------------------------------------
template <typename T>
cudaError_t launch_step(const Geom& g, int order, const WaveFields<T>& f, StepMode mode,
                        const StepScalars& s, cudaStream_t st, long long* nlaunch);
template <typename T>
cudaError_t launch_minvK(const Geom& g, int order, const T* u, T* out, const T* lam,
                         const T* mu, const T* irh2, T* sigma, cudaStream_t st, long long* nlaunch,
                         const T* met = nullptr);

// ---- vector kernels (ewh_krylov.cu) -----------------------------------------
// dense FP64 [rhs][comp][unknowns] <-> padded T
template <typename T>
cudaError_t launch_pack(const Geom& g, const double* dense, T* padded, cudaStream_t st);
template <typename T>
cudaError_t launch_unpack(const Geom& g, const T* padded, double* dense, const double* sub_from,
                          cudaStream_t st);
// Fused CG direction update and pack: p = r + beta_r p (per rhs), padded = (T) p.
template <typename T>
cudaError_t launch_pupdate_pack(const Geom& g, const double* r, double* p, const double* beta,
                                T* padded, cudaStream_t st);

// Deterministic M inner products: partial sums into part[rhs][nblk], then
// a fixed-order second pass.
int dot_blocks(const Geom& g);
cudaError_t launch_mdot_partial(const Geom& g, const double* mw, const double* x, const double* y,
                                double* part, cudaStream_t st);
cudaError_t launch_mdot_final(const Geom& g, const double* part, double* out, cudaStream_t st);

// CG pieces (all scalars per rhs live on the device):
//   alpha = active ? rr / pq : 0  (sets breakdown flag if pq <= 0)
cudaError_t launch_cg_alpha(int nrhs, const double* pq_part, int nblk, const double* rr,
                            double* alpha, int* active, int* flags, cudaStream_t st);
//   x += alpha p ; r -= alpha q ; partial (r, r)_M
cudaError_t launch_cg_xr_update(const Geom& g, const double* mw, const double* alpha, const double* p,
                                const double* q, double* x, double* r, double* part, cudaStream_t st);
//   rr_new = sum part ; beta = rr_new / rr ; rr = rr_new ; res = sqrt(rr_new / bb)
cudaError_t launch_cg_beta(int nrhs, const double* part, int nblk, double* rr, const double* bb,
                           double* beta, double* res, const int* active, cudaStream_t st);
//   device-side loop control after an iteration (a while-conditional graph
//   node): ++ctl[0], hist[ctl[0] - 1] = max active res, continue unless a
//   replacement is due (anchor: nrhs anchors, then tol and drop), the
//   breakdown flag is set or ctl[0] reaches ctl[1]
cudaError_t launch_cg_control(cudaGraphConditionalHandle h, int nrhs, const double* res, const int* active,
                              const double* anchor, const int* flags, int* ctl, double* hist, cudaStream_t st);
//   after a residual replacement: beta *= dot / rr ; rr = dot ; res = sqrt(dot / bb)
cudaError_t launch_cg_replace(int nrhs, const double* dot, double* rr, double* beta, double* res, const double* bb,
                              cudaStream_t st);
// conjugate residual: res = sqrt((r,r)_M / bb); beta = (r,Ar)_new/(r,Ar)_old;
// p = r + beta p, Ap = Ar + beta Ap
cudaError_t launch_res(int nrhs, const double* part, int nblk, const double* bb, double* res, const int* active,
                       cudaStream_t st);
cudaError_t launch_cr_beta(int nrhs, const double* part, int nblk, double* rar, double* beta, const int* active,
                           int init, cudaStream_t st);
cudaError_t launch_cr_pupdate(const Geom& g, const double* r, const double* ar, double* p, double* ap,
                              const double* beta, cudaStream_t st);
cudaError_t launch_axpby(long long n, double a, const double* x, double b, double* y, cudaStream_t st);
cudaError_t launch_fill_mass(const Geom& g, int order, const double* rho_full, double h, double* mw,
                             cudaStream_t st);
// mapped grids: 6 dense planes (y_r, -x_r, -y_q, x_q, 1/J, J) of n0*n1 nodes
cudaError_t launch_curv_metrics(int n0, int n1, double h, const double* X, const double* Y, double* out,
                                cudaStream_t st);

// ---- on-chip resident wave solve (ewh_stencil.cu) --------------------------
// Order 4 (SBP), 2D, FP32, one right-hand side: all nt*periods time levels in
// one cooperative launch, one CTA per SM, each owning a bx x by block of
// nodes whose state stays in shared memory and registers.  Shapes: threads
// per CTA x pairs of regular own nodes (adjacent along x) per thread at most.
constexpr int RS_SHAPES = 3;
constexpr int RS_SHAPE_THREADS[RS_SHAPES] = {1024, 768, 512};
constexpr int RS_SHAPE_PAIRS[RS_SHAPES] = {4, 5, 7};
struct ResidentPlan {
  int ok = 0;
  int shape = 0;       // index into RS_SHAPE_*
  int px = 0, py = 0;  // CTAs per axis
  int bx = 0, by = 0;  // node block per CTA (the last block per axis may be smaller, >= 8)
  int ex = 0;          // width of the first block along x (the x-closure columns cost more, so the
                       // first and last blocks along x are narrower); the last is the remainder
  size_t smem = 0;     // dynamic shared memory per CTA in bytes
  int rg = 1;          // right-hand sides per cooperative launch (rg x px x py CTAs, all co-resident)
  int groups = 1;      // launches per wave solve, one after another
};
// Partition of g for the current device and a CTA shape (ok = 0 when g does
// not fit on chip).
ResidentPlan plan_resident_o4(const Geom& g, int shape);
struct ResidentIO {
  const float* u0;      // u^0 (padded, 2 components)
  float* xbuf0;         // exchange buffers for the rims of u (padded, 2 components)
  float* xbuf1;
  float* acc;           // filter accumulator, written at the end (unknowns only)
  const float* lam;
  const float* mu;
  const float* irh2;
  const float* frho;    // null: unforced
  const double* cosn;   // [nsteps] cos(w t_n)
  const double* wnew;   // [nsteps] trapezoid weight of level n+1
  double kt;            // c dt^2
  double w0;            // trapezoid weight of level 0
  int nsteps;
  unsigned* bar;        // [8]: [0] grid-barrier arrivals and [1] error flag (both zeroed by the
                        // launcher); [2..3] the barrier-wait limit in ns (u64, 0 = give up at
                        // once); [4] launches whose wait gave up (never reset by a launch)
};
constexpr int RS_BAR_WORDS = 8;
constexpr unsigned long long RS_WAIT_NS_DEFAULT = 1000000000ull;  // one barrier wait, 1 s
cudaError_t launch_resident_o4(const Geom& g, const ResidentPlan& p, const ResidentIO& io, cudaStream_t st);

// ---- fused 3D order-4 FP32 step (ewh_zmarch.cu) ------------------------------
ZmPlan plan_zmarch(const Geom& g, const float* u_a, const float* u_b, unsigned* ctl);
cudaError_t launch_zmarch(const Geom& g, const ZmPlan& p, int shape, const WaveFields<float>& f, StepMode mode,
                          const StepScalars& s, cudaStream_t st);

// ---- fused 2D order-4 FP32 step (ewh_ymarch.cu) ------------------------------
// Step-kernel variant of the 2D order-4 FP32 launcher that runs it (after
// the split tiles 0..3, the fused kernel 4 and the resident shapes 5..7).
constexpr int YM_VARIANT = 8;
ZmPlan plan_ymarch(const Geom& g, const float* u_a, const float* u_b, unsigned* ctl);
cudaError_t launch_ymarch(const Geom& g, const ZmPlan& p, const WaveFields<float>& f, StepMode mode,
                          const StepScalars& s, cudaStream_t st);

// Message for ewh_last_error(NULL) of calls that have no context.
void set_global_error(const std::string& msg);

}  // namespace ewh
