// Fused leapfrog + trapezoid-filter step kernels.
//
// One launch advances every right-hand side by one time level of the
// time-corrected explicit scheme (Section 4.3, eq. elastic-time-explicit-
// corrected), written in increment form
//     delta^{n+1} = delta^n - kt (M^{-1} K u^n + (f / rho) cos(w t_n)),
//     u^{n+1}     = u^n + delta^{n+1},
//     acc        += w_{n+1} u^{n+1}                (trapezoid filter, eq. qoper)
// with the Taylor start folded into the first launch:
//     delta^1 = -(kt/2) (M^{-1} K u^0 + f / rho),  acc = w_0 u^0 + w_1 u^1.
// K = -L_h is the Hessian of the discrete elastic energy (Section 4.1):
//   order 2: compact form; pure terms on edges with edge coefficients equal
//            to the mean of the two end nodes, mixed terms at nodes with
//            centred differences (one-sided on a free boundary node), the
//            trapezoid factor 1/2 per free side;
//   order 4: pointwise energy density with all first derivatives from the
//            fourth-order diagonal-norm summation-by-parts operator D; then
//            M^{-1} K u = (1/(rho h^2)) sum_a [ -D_a sigma_{.a} + H_a^{-1} B_a sigma_{.a} ].
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "ewh_internal.cuh"

namespace ewh {

// The SBP boundary closure (SBP_CLOSURE) in constant memory.
#define EWH_SBP_ROW(T, r)                                                                         \
  {                                                                                               \
    (T)SBP_CLOSURE[r][0], (T)SBP_CLOSURE[r][1], (T)SBP_CLOSURE[r][2], (T)SBP_CLOSURE[r][3],        \
        (T)SBP_CLOSURE[r][4], (T)SBP_CLOSURE[r][5]                                                \
  }
__constant__ double c_sbp_d[4][6] = {EWH_SBP_ROW(double, 0), EWH_SBP_ROW(double, 1), EWH_SBP_ROW(double, 2),
                                     EWH_SBP_ROW(double, 3)};
__constant__ float c_sbp_f[4][6] = {EWH_SBP_ROW(float, 0), EWH_SBP_ROW(float, 1), EWH_SBP_ROW(float, 2),
                                    EWH_SBP_ROW(float, 3)};
#undef EWH_SBP_ROW

template <typename T>
__device__ __forceinline__ T sbp_coef(int r, int j);
template <>
__device__ __forceinline__ double sbp_coef<double>(int r, int j) { return c_sbp_d[r][j]; }
template <>
__device__ __forceinline__ float sbp_coef<float>(int r, int j) { return c_sbp_f[r][j]; }

// SBP first derivative along one axis at position p of a line of N nodes;
// v points at the node, s is the element stride along the axis.
template <typename T>
__device__ __forceinline__ T sbp_d1(const T* v, long long s, int p, int N) {
  if (p < 4) {
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < 6; ++j) acc += sbp_coef<T>(p, j) * v[(long long)(j - p) * s];
    return acc;
  }
  if (p > N - 5) {
    const int r = N - 1 - p;
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < 6; ++j) acc -= sbp_coef<T>(r, j) * v[(long long)(r - j) * s];
    return acc;
  }
  return (v[-2 * s] - T(8) * v[-s] + T(8) * v[s] - v[2 * s]) * T(1.0 / 12.0);
}

// interior row of the SBP first derivative (unit spacing): (1, -8, 0, 8, -1) / 12
template <typename T>
__device__ __forceinline__ T c4(T m2, T m1, T p1, T p2) {
  return (m2 - T(8) * m1 + T(8) * p1 - p2) * T(1.0 / 12.0);
}

// Programmatic dependent launch: a step kernel may start while the previous
// one drains.  Before pdl_wait() a kernel reads only data the solve never
// writes (lambda, mu, 1/(rho h^2), f/rho); pdl_wait() returns once the previous
// kernel has completed and its writes are visible; pdl_trigger() lets the next
// kernel begin launching.  Both are no-ops for a normal launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Time update shared by all kernels.  a = M^{-1} K u (FP of the state).
// ---------------------------------------------------------------------------
template <typename T, int MODE, bool FORCED>
__device__ __forceinline__ void leapfrog_update(const WaveFields<T>& f, long long p, T uval, T a,
                                                const StepScalars& s) {
  if (MODE == 3) {  // operator only
    f.u_next[p] = a;
    return;
  }
  if (FORCED) a += f.frho[p] * T(s.cosn);
  if (MODE == STEP_FIRST) {
    const T d = T(-0.5) * T(s.kt) * a;
    const T un = uval + d;
    f.delta[p] = d;
    f.u_next[p] = un;
    f.acc[p] = T(s.w0) * uval + T(s.wnew) * un;
  } else {
    const T d = f.delta[p] - T(s.kt) * a;
    const T un = uval + d;
    if (MODE == STEP_MID) {
      f.delta[p] = d;
      f.u_next[p] = un;
    }
    f.acc[p] += T(s.wnew) * un;
  }
}

// The same update with delta^n, acc and f/rho already loaded (dprev, accprev
// are not read at the first level; fr only when FORCED).
template <typename T, int MODE, bool FORCED>
__device__ __forceinline__ void leapfrog_update_pre(const WaveFields<T>& f, long long p, T uval, T a,
                                                    const StepScalars& s, T dprev, T accprev, T fr) {
  if (MODE == 3) {
    f.u_next[p] = a;
    return;
  }
  if (FORCED) a += fr * T(s.cosn);
  if (MODE == STEP_FIRST) {
    const T d = T(-0.5) * T(s.kt) * a;
    const T un = uval + d;
    f.delta[p] = d;
    f.u_next[p] = un;
    f.acc[p] = T(s.w0) * uval + T(s.wnew) * un;
  } else {
    const T d = dprev - T(s.kt) * a;
    const T un = uval + d;
    if (MODE == STEP_MID) {
      f.delta[p] = d;
      f.u_next[p] = un;
    }
    f.acc[p] = accprev + T(s.wnew) * un;
  }
}


// ---------------------------------------------------------------------------
// Order 2, 2D: 32 x 8 tile, one node per thread, halo 1 in shared memory.
// ---------------------------------------------------------------------------
template <typename T, int MODE, bool FORCED, int TYV>
__global__ void __launch_bounds__(32 * TYV) step2d_o2(Geom g, WaveFields<T> f, StepScalars s) {
  if (g.dim != 2) return;
  pdl_wait();
  pdl_trigger();
  constexpr int TX = 32, TY = TYV, SX = TX + 2, SY = TY + 2;
  __shared__ T su[2][SY][SX];
  __shared__ T sl[SY][SX];
  __shared__ T sm[SY][SX];
  const int rhs = blockIdx.z;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int tid = threadIdx.y * TX + threadIdx.x;
  for (int i = tid; i < SX * SY; i += TX * TY) {
    const int lx = i % SX, ly = i / SX;
    const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
    const long long pu = pidx(g, rhs, 0, gx, gy, 0);
    su[0][ly][lx] = f.u_cur[pu];
    su[1][ly][lx] = f.u_cur[pu + g.field];
    const long long pc = pidx(g, 0, 0, gx, gy, 0);
    sl[ly][lx] = f.lam[pc];
    sm[ly][lx] = f.mu[pc];
  }
  __syncthreads();
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
  if (!is_unknown(g, x, y, 0)) return;
  const int tx = threadIdx.x + 1, ty = threadIdx.y + 1;
  const int nx = g.n[0], ny = g.n[1];
  // at an unknown node, sitting on the first/last grid line means a free side
  const bool fxl = (x == 0), fxh = (x == nx - 1), fyl = (y == 0), fyh = (y == ny - 1);

  auto U = [&](int c, int dx, int dy) -> T { return su[c][ty + dy][tx + dx]; };
  auto L = [&](int dx, int dy) -> T { return sl[ty + dy][tx + dx]; };
  auto M = [&](int dx, int dy) -> T { return sm[ty + dy][tx + dx]; };
  auto coef = [&](bool p_wave, int dx, int dy) -> T {
    return p_wave ? L(dx, dy) + T(2) * M(dx, dy) : M(dx, dy);
  };
  // pure terms (edges), already divided by the trapezoid factor of the node
  auto pureX = [&](int c, bool p_wave) -> T {
    const T c0 = coef(p_wave, 0, 0);
    T t = T(0);
    if (x > 0) t += T(0.5) * (c0 + coef(p_wave, -1, 0)) * (U(c, 0, 0) - U(c, -1, 0));
    if (x < nx - 1) t -= T(0.5) * (c0 + coef(p_wave, 1, 0)) * (U(c, 1, 0) - U(c, 0, 0));
    return (fxl || fxh) ? T(2) * t : t;
  };
  auto pureY = [&](int c, bool p_wave) -> T {
    const T c0 = coef(p_wave, 0, 0);
    T t = T(0);
    if (y > 0) t += T(0.5) * (c0 + coef(p_wave, 0, -1)) * (U(c, 0, 0) - U(c, 0, -1));
    if (y < ny - 1) t -= T(0.5) * (c0 + coef(p_wave, 0, 1)) * (U(c, 0, 1) - U(c, 0, 0));
    return (fyl || fyh) ? T(2) * t : t;
  };
  // centred differences at the node offset by dx (resp. dy)
  auto CyAt = [&](int c, int dx) -> T {
    if (fyh) return U(c, dx, 0) - U(c, dx, -1);
    if (fyl) return U(c, dx, 1) - U(c, dx, 0);
    return T(0.5) * (U(c, dx, 1) - U(c, dx, -1));
  };
  auto CxAt = [&](int c, int dy) -> T {
    if (fxh) return U(c, 0, dy) - U(c, -1, dy);
    if (fxl) return U(c, 1, dy) - U(c, 0, dy);
    return T(0.5) * (U(c, 1, dy) - U(c, -1, dy));
  };
  // transposed centred difference (divided by the node's trapezoid factor)
  auto Gx = [&](bool use_lam, int c, int dx) -> T {
    if (!is_unknown(g, x + dx, y, 0)) return T(0);
    return (use_lam ? L(dx, 0) : M(dx, 0)) * CyAt(c, dx);
  };
  auto Gy = [&](bool use_lam, int c, int dy) -> T {
    if (!is_unknown(g, x, y + dy, 0)) return T(0);
    return (use_lam ? L(0, dy) : M(0, dy)) * CxAt(c, dy);
  };
  auto Zx = [&](bool use_lam, int c) -> T {
    if (fxh) return Gx(use_lam, c, -1) + Gx(use_lam, c, 0);
    if (fxl) return -(Gx(use_lam, c, 0) + Gx(use_lam, c, 1));
    return T(0.5) * (Gx(use_lam, c, -1) - Gx(use_lam, c, 1));
  };
  auto Zy = [&](bool use_lam, int c) -> T {
    if (fyh) return Gy(use_lam, c, -1) + Gy(use_lam, c, 0);
    if (fyl) return -(Gy(use_lam, c, 0) + Gy(use_lam, c, 1));
    return T(0.5) * (Gy(use_lam, c, -1) - Gy(use_lam, c, 1));
  };
  // K u for u (x-displacement) and v (y-displacement)
  const T Ku = pureX(0, true) + pureY(0, false) + Zx(true, 1) + Zy(false, 1);
  const T Kv = pureX(1, false) + pureY(1, true) + Zy(true, 0) + Zx(false, 0);
  const T irh = f.irh2[pidx(g, 0, 0, x, y, 0)];
  const long long p0 = pidx(g, rhs, 0, x, y, 0);
  leapfrog_update<T, MODE, FORCED>(f, p0, U(0, 0, 0), Ku * irh, s);
  leapfrog_update<T, MODE, FORCED>(f, p0 + g.field, U(1, 0, 0), Kv * irh, s);
}

// ---------------------------------------------------------------------------
// Order 2, 3D: 32 x 4 x 2 tile, halo 1.
// ---------------------------------------------------------------------------
template <typename T, int MODE, bool FORCED>
__global__ void __launch_bounds__(256) step3d_o2(Geom g, WaveFields<T> f, StepScalars s) {
  if (g.dim != 3) return;
  pdl_wait();
  pdl_trigger();
  constexpr int TX = 32, TY = 4, TZ = 2, SX = TX + 2, SY = TY + 2, SZ = TZ + 2;
  __shared__ T su[3][SZ][SY][SX];
  __shared__ T sl[SZ][SY][SX];
  __shared__ T sm[SZ][SY][SX];
  const int nzb = (g.n[2] + TZ - 1) / TZ;
  const int rhs = blockIdx.z / nzb;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = (blockIdx.z % nzb) * TZ;
  const int tid = (threadIdx.z * TY + threadIdx.y) * TX + threadIdx.x;
  for (int i = tid; i < SX * SY * SZ; i += TX * TY * TZ) {
    const int lx = i % SX, ly = (i / SX) % SY, lz = i / (SX * SY);
    const int gx = x0 - 1 + lx, gy = y0 - 1 + ly, gz = z0 - 1 + lz;
    const long long pu = pidx(g, rhs, 0, gx, gy, gz);
    su[0][lz][ly][lx] = f.u_cur[pu];
    su[1][lz][ly][lx] = f.u_cur[pu + g.field];
    su[2][lz][ly][lx] = f.u_cur[pu + 2 * g.field];
    const long long pc = pidx(g, 0, 0, gx, gy, gz);
    sl[lz][ly][lx] = f.lam[pc];
    sm[lz][ly][lx] = f.mu[pc];
  }
  __syncthreads();
  const int pos[3] = {x0 + (int)threadIdx.x, y0 + (int)threadIdx.y, z0 + (int)threadIdx.z};
  if (!is_unknown(g, pos[0], pos[1], pos[2])) return;
  const int t0[3] = {(int)threadIdx.x + 1, (int)threadIdx.y + 1, (int)threadIdx.z + 1};
  const bool lo[3] = {pos[0] == 0, pos[1] == 0, pos[2] == 0};
  const bool hi[3] = {pos[0] == g.n[0] - 1, pos[1] == g.n[1] - 1, pos[2] == g.n[2] - 1};

  auto U = [&](int c, int dx, int dy, int dz) -> T { return su[c][t0[2] + dz][t0[1] + dy][t0[0] + dx]; };
  auto L = [&](int dx, int dy, int dz) -> T { return sl[t0[2] + dz][t0[1] + dy][t0[0] + dx]; };
  auto Mu = [&](int dx, int dy, int dz) -> T { return sm[t0[2] + dz][t0[1] + dy][t0[0] + dx]; };
  auto Uo = [&](int c, const int* o) -> T { return U(c, o[0], o[1], o[2]); };

  T Kc[3];
#pragma unroll
  for (int al = 0; al < 3; ++al) {
    T acc = T(0);
    // pure terms along every axis
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      int e[3] = {0, 0, 0};
      e[a] = 1;
      const T c0 = (al == a) ? L(0, 0, 0) + T(2) * Mu(0, 0, 0) : Mu(0, 0, 0);
      T t = T(0);
      if (pos[a] > 0) {
        const T cl = (al == a) ? L(-e[0], -e[1], -e[2]) + T(2) * Mu(-e[0], -e[1], -e[2]) : Mu(-e[0], -e[1], -e[2]);
        t += T(0.5) * (c0 + cl) * (U(al, 0, 0, 0) - U(al, -e[0], -e[1], -e[2]));
      }
      if (pos[a] < g.n[a] - 1) {
        const T cr = (al == a) ? L(e[0], e[1], e[2]) + T(2) * Mu(e[0], e[1], e[2]) : Mu(e[0], e[1], e[2]);
        t -= T(0.5) * (c0 + cr) * (U(al, e[0], e[1], e[2]) - U(al, 0, 0, 0));
      }
      acc += (lo[a] || hi[a]) ? T(2) * t : t;
    }
    // mixed terms: for each beta != alpha
    //   Z_alpha( lambda C_beta u_beta ) + Z_beta( mu C_alpha u_beta )
#pragma unroll
    for (int be = 0; be < 3; ++be) {
      if (be == al) continue;
#pragma unroll
      for (int term = 0; term < 2; ++term) {
        const int za = term == 0 ? al : be;   // axis of the transposed difference
        const int cb = term == 0 ? be : al;   // axis of the inner difference
        auto G = [&](int k) -> T {
          int o[3] = {0, 0, 0};
          o[za] = k;
          if (!is_unknown(g, pos[0] + o[0], pos[1] + o[1], pos[2] + o[2])) return T(0);
          int op[3] = {o[0], o[1], o[2]}, om[3] = {o[0], o[1], o[2]};
          op[cb] += 1;
          om[cb] -= 1;
          T d;
          if (hi[cb]) d = Uo(be, o) - Uo(be, om);
          else if (lo[cb]) d = Uo(be, op) - Uo(be, o);
          else d = T(0.5) * (Uo(be, op) - Uo(be, om));
          const T cf = term == 0 ? L(o[0], o[1], o[2]) : Mu(o[0], o[1], o[2]);
          return cf * d;
        };
        T z;
        if (hi[za]) z = G(-1) + G(0);
        else if (lo[za]) z = -(G(0) + G(1));
        else z = T(0.5) * (G(-1) - G(1));
        acc += z;
      }
    }
    Kc[al] = acc;
  }
  const T irh = f.irh2[pidx(g, 0, 0, pos[0], pos[1], pos[2])];
  const long long p0 = pidx(g, rhs, 0, pos[0], pos[1], pos[2]);
#pragma unroll
  for (int al = 0; al < 3; ++al)
    leapfrog_update<T, MODE, FORCED>(f, p0 + al * g.field, U(al, 0, 0, 0), Kc[al] * irh, s);
}

// ---------------------------------------------------------------------------
// Order 4 (SBP), any dimension: stress pass then divergence + update pass.
// Stress fields per rhs: 2D (xx, yy, xy); 3D (xx, yy, zz, xy, xz, yz).
// ---------------------------------------------------------------------------
template <int DIM>
__host__ __device__ constexpr int nsig() { return DIM == 2 ? 3 : 6; }
template <int DIM>
__device__ __forceinline__ int sig_index(int a, int b) {
  if (a == b) return a;
  if (DIM == 2) return 2;
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  return lo == 0 ? (hi == 1 ? 3 : 4) : 5;
}

// 3D order 4: the 32 x 8 block of this z plane and its 2-node reach lie in
// rows, columns and planes 4 .. n - 5 (every difference central, every node
// an unknown): uniform per block, so the fast path never diverges.
__device__ __forceinline__ bool o4_3d_inner(const Geom& g, int z) {
  const int x0 = blockIdx.x * blockDim.x, y0 = blockIdx.y * blockDim.y;
  return x0 >= 4 && x0 + (int)blockDim.x - 1 <= g.n[0] - 5 && y0 >= 4 && y0 + (int)blockDim.y - 1 <= g.n[1] - 5 &&
         z >= 4 && z <= g.n[2] - 5;
}

template <typename T, int DIM>
__global__ void __launch_bounds__(256) sbp_stress(Geom g, const T* __restrict__ u, const T* __restrict__ lam,
                                                  const T* __restrict__ mu, T* __restrict__ sig) {
  if (g.dim != DIM) return;  // launched for the wrong dimension: touch nothing
  pdl_wait();
  pdl_trigger();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  int z = 0, rhs = blockIdx.z;
  if (DIM == 3) {
    const int nz = g.n[2];
    z = blockIdx.z % nz;
    rhs = blockIdx.z / nz;
  }
  if (x >= g.n[0] || y >= g.n[1]) return;
  if (DIM == 3 && o4_3d_inner(g, z)) {  // central differences only, 32-bit offsets from one base
    const int sy = g.np[0], sz = (int)g.plane;  // neighbour offsets: 2 planes index in 32 bits
    const long long fld = g.field;
    const long long pc = pidx(g, 0, 0, x, y, z);
    const T* U = u + pidx(g, rhs, 0, x, y, z);
    T gr[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T* b = U + c * fld;
      gr[c][0] = c4(b[-2], b[-1], b[1], b[2]);
      gr[c][1] = c4(b[-2 * sy], b[-sy], b[sy], b[2 * sy]);
      gr[c][2] = c4(b[-2 * sz], b[-sz], b[sz], b[2 * sz]);
    }
    const T l = lam[pc], m = mu[pc];
    const T div = gr[0][0] + gr[1][1] + gr[2][2];
    T* o = sig + (long long)rhs * 6 * g.field + pc;
    o[0] = l * div + T(2) * m * gr[0][0];
    o[fld] = l * div + T(2) * m * gr[1][1];
    o[2 * fld] = l * div + T(2) * m * gr[2][2];
    o[3 * fld] = m * (gr[0][1] + gr[1][0]);
    o[4 * fld] = m * (gr[0][2] + gr[2][0]);
    o[5 * fld] = m * (gr[1][2] + gr[2][1]);
    return;
  }
  const int pos[3] = {x, y, z};
  const long long stride[3] = {1, (long long)g.np[0], g.plane};
  // gradient grad[alpha][a] = D_a u_alpha
  T grad[DIM][DIM];
#pragma unroll
  for (int al = 0; al < DIM; ++al) {
    const T* base = u + pidx(g, rhs, al, x, y, z);
#pragma unroll
    for (int a = 0; a < DIM; ++a) grad[al][a] = sbp_d1<T>(base, stride[a], pos[a], g.n[a]);
  }
  const long long pc = pidx(g, 0, 0, x, y, z);
  const T l = lam[pc], m = mu[pc];
  T div = T(0);
#pragma unroll
  for (int a = 0; a < DIM; ++a) div += grad[a][a];
  T* out = sig + (long long)rhs * nsig<DIM>() * g.field + (pc - 0);
#pragma unroll
  for (int a = 0; a < DIM; ++a) out[(long long)a * g.field] = l * div + T(2) * m * grad[a][a];
#pragma unroll
  for (int a = 0; a < DIM; ++a)
#pragma unroll
    for (int b = a + 1; b < DIM; ++b)
      out[(long long)sig_index<DIM>(a, b) * g.field] = m * (grad[a][b] + grad[b][a]);
}

template <typename T, int DIM, int MODE, bool FORCED>
__global__ void __launch_bounds__(256) sbp_divergence_step(Geom g, WaveFields<T> f, StepScalars s) {
  if (g.dim != DIM) return;
  pdl_wait();
  pdl_trigger();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  int z = 0, rhs = blockIdx.z;
  if (DIM == 3) {
    const int nz = g.n[2];
    z = blockIdx.z % nz;
    rhs = blockIdx.z / nz;
  }
  if (DIM == 3 && x < g.n[0] && y < g.n[1] && o4_3d_inner(g, z)) {  // central differences, no boundary terms
    const int sy = g.np[0], sz = (int)g.plane;  // neighbour offsets: 2 planes index in 32 bits
    const long long fld = g.field;
    const long long pc = pidx(g, 0, 0, x, y, z);
    const T* S = f.sigma + (long long)rhs * 6 * g.field + pc;  // planes xx, yy, zz, xy, xz, yz
    const T* Sxx = S;
    const T* Syy = S + fld;
    const T* Szz = S + 2 * fld;
    const T* Sxy = S + 3 * fld;
    const T* Sxz = S + 4 * fld;
    const T* Syz = S + 5 * fld;
    const T ku = -(c4(Sxx[-2], Sxx[-1], Sxx[1], Sxx[2]) + c4(Sxy[-2 * sy], Sxy[-sy], Sxy[sy], Sxy[2 * sy]) +
                   c4(Sxz[-2 * sz], Sxz[-sz], Sxz[sz], Sxz[2 * sz]));
    const T kv = -(c4(Sxy[-2], Sxy[-1], Sxy[1], Sxy[2]) + c4(Syy[-2 * sy], Syy[-sy], Syy[sy], Syy[2 * sy]) +
                   c4(Syz[-2 * sz], Syz[-sz], Syz[sz], Syz[2 * sz]));
    const T kw = -(c4(Sxz[-2], Sxz[-1], Sxz[1], Sxz[2]) + c4(Syz[-2 * sy], Syz[-sy], Syz[sy], Syz[2 * sy]) +
                   c4(Szz[-2 * sz], Szz[-sz], Szz[sz], Szz[2 * sz]));
    const T irh = f.irh2[pc];
    const long long p0 = pidx(g, rhs, 0, x, y, z);
    leapfrog_update<T, MODE, FORCED>(f, p0, f.u_cur[p0], ku * irh, s);
    leapfrog_update<T, MODE, FORCED>(f, p0 + fld, f.u_cur[p0 + fld], kv * irh, s);
    leapfrog_update<T, MODE, FORCED>(f, p0 + 2 * fld, f.u_cur[p0 + 2 * fld], kw * irh, s);
    return;
  }
  if (!is_unknown(g, x, y, z)) return;
  const int pos[3] = {x, y, z};
  const long long stride[3] = {1, (long long)g.np[0], g.plane};
  const long long pc = pidx(g, 0, 0, x, y, z);
  const T* sig = f.sigma + (long long)rhs * nsig<DIM>() * g.field + pc;
  const T inv_h0 = T(48.0 / 17.0);
  const T irh = f.irh2[pc];
  const long long p0 = pidx(g, rhs, 0, x, y, z);
#pragma unroll
  for (int al = 0; al < DIM; ++al) {
    T k = T(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const T* sa = sig + (long long)sig_index<DIM>(al, a) * g.field;
      k -= sbp_d1<T>(sa, stride[a], pos[a], g.n[a]);
      if (pos[a] == 0) k -= inv_h0 * sa[0];                 // free low side
      else if (pos[a] == g.n[a] - 1) k += inv_h0 * sa[0];   // free high side
    }
    const long long p = p0 + al * g.field;
    leapfrog_update<T, MODE, FORCED>(f, p, f.u_cur[p], k * irh, s);
  }
}

// ---------------------------------------------------------------------------
// Order 4 (SBP), 2D, split into two launches (stresses, then divergence and
// update), one node per thread, 32 x 8 blocks.  Blocks whose nodes and stencil
// reach lie inside the grid away from every SBP closure row stage their
// operands (tile + 2-node halo) in shared memory with a few independent
// coalesced loads per thread and difference them there; blocks near a side
// run the generic per-node code from global memory.
// ---------------------------------------------------------------------------
constexpr int TL_H = 2;

// 12 times the interior difference: the order-4 kernels that carry the
// operator as 12 D (stresses 12 sigma, divergence 144 D sigma) apply the
// 1 / 144 once per node, with 1 / (rho h^2), instead of once per difference.
template <typename T>
__device__ __forceinline__ T c4u(T m2, T m1, T p1, T p2) {
  return m2 - T(8) * m1 + T(8) * p1 - p2;
}

// every node of the block and its 2-node reach lies in rows/columns 4..N-5
template <int TL_TX, int TL_TY>
__device__ __forceinline__ bool tl_block_interior(const Geom& g, int x0, int y0) {
  return x0 >= 4 && x0 + TL_TX - 1 <= g.n[0] - 5 && y0 >= 4 && y0 + TL_TY - 1 <= g.n[1] - 5;
}

template <typename T>
__device__ __forceinline__ void stress2d_node(const Geom& g, const T* u, const T* lam, const T* mu, T* sig, int rhs,
                                              int x, int y) {
  const long long sy = g.np[0];
  const T* U = u + pidx(g, rhs, 0, x, y, 0);
  const T* V = U + g.field;
  const T u_x = sbp_d1<T>(U, 1, x, g.n[0]);
  const T u_y = sbp_d1<T>(U, sy, y, g.n[1]);
  const T v_x = sbp_d1<T>(V, 1, x, g.n[0]);
  const T v_y = sbp_d1<T>(V, sy, y, g.n[1]);
  const long long pc = pidx(g, 0, 0, x, y, 0);
  const T l = lam[pc], m = mu[pc];
  const T div = u_x + v_y;
  T* out = sig + (long long)rhs * 3 * g.field + pc;  // 12 sigma, as the interior tiles store it
  out[0] = T(12) * (l * div + T(2) * m * u_x);
  out[g.field] = T(12) * (l * div + T(2) * m * v_y);
  out[2 * g.field] = T(12) * (m * (u_y + v_x));
}

template <typename T, int TL_TX, int TL_TY>
__global__ void __launch_bounds__(TL_TX * TL_TY) sbp_stress2d_tl(Geom g, const T* __restrict__ u,
                                                                 const T* __restrict__ lam, const T* __restrict__ mu,
                                                                 T* __restrict__ sig) {
  if (g.dim != 2) return;
  constexpr int SX = TL_TX + 2 * TL_H, SY = TL_TY + 2 * TL_H;
  __shared__ T su[2][SY][SX];
  const int rhs = blockIdx.z;
  const int x0 = blockIdx.x * TL_TX, y0 = blockIdx.y * TL_TY;
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
  if (!tl_block_interior<TL_TX, TL_TY>(g, x0, y0)) {  // uniform per block
    pdl_wait();
    pdl_trigger();
    if (x < g.n[0] && y < g.n[1]) stress2d_node<T>(g, u, lam, mu, sig, rhs, x, y);
    return;
  }
  const long long pc = pidx(g, 0, 0, x, y, 0);
  const T l = lam[pc], m = mu[pc];               // static: read before the wait
  pdl_wait();
  pdl_trigger();
  const T* U = u + pidx(g, rhs, 0, x0 - TL_H, y0 - TL_H, 0);
  const int tid = threadIdx.y * TL_TX + threadIdx.x;
  for (int i = tid; i < SX * SY; i += TL_TX * TL_TY) {
    const int lx = i % SX, ly = i / SX;
    const long long off = (long long)ly * g.np[0] + lx;
    su[0][ly][lx] = U[off];
    su[1][ly][lx] = U[off + g.field];
  }
  __syncthreads();
  const int cx = threadIdx.x + TL_H, cy = threadIdx.y + TL_H;
  // 12 D u and 12 sigma
  const T u_x = c4u(su[0][cy][cx - 2], su[0][cy][cx - 1], su[0][cy][cx + 1], su[0][cy][cx + 2]);
  const T v_x = c4u(su[1][cy][cx - 2], su[1][cy][cx - 1], su[1][cy][cx + 1], su[1][cy][cx + 2]);
  const T u_y = c4u(su[0][cy - 2][cx], su[0][cy - 1][cx], su[0][cy + 1][cx], su[0][cy + 2][cx]);
  const T v_y = c4u(su[1][cy - 2][cx], su[1][cy - 1][cx], su[1][cy + 1][cx], su[1][cy + 2][cx]);
  const T div = u_x + v_y;
  T* out = sig + (long long)rhs * 3 * g.field + pc;
  out[0] = l * div + T(2) * m * u_x;
  out[g.field] = l * div + T(2) * m * v_y;
  out[2 * g.field] = m * (u_y + v_x);
}

template <typename T, int MODE, bool FORCED>
__device__ __forceinline__ void div2d_node(const Geom& g, const WaveFields<T>& f, const StepScalars& s, int rhs, int x,
                                           int y) {
  if (!is_unknown(g, x, y, 0)) return;
  const long long sy = g.np[0];
  const long long pc = pidx(g, 0, 0, x, y, 0);
  const T* sg = f.sigma + (long long)rhs * 3 * g.field + pc;
  const T* sxx = sg;
  const T* syy = sg + g.field;
  const T* sxy = sg + 2 * g.field;
  T ku = -sbp_d1<T>(sxx, 1, x, g.n[0]) - sbp_d1<T>(sxy, sy, y, g.n[1]);
  T kv = -sbp_d1<T>(sxy, 1, x, g.n[0]) - sbp_d1<T>(syy, sy, y, g.n[1]);
  const T inv_h0 = T(48.0 / 17.0);
  if (x == 0) {
    ku -= inv_h0 * sxx[0];
    kv -= inv_h0 * sxy[0];
  } else if (x == g.n[0] - 1) {
    ku += inv_h0 * sxx[0];
    kv += inv_h0 * sxy[0];
  }
  if (y == 0) {
    ku -= inv_h0 * sxy[0];
    kv -= inv_h0 * syy[0];
  } else if (y == g.n[1] - 1) {
    ku += inv_h0 * sxy[0];
    kv += inv_h0 * syy[0];
  }
  const T irh = f.irh2[pc] * T(1.0 / 12.0);  // the scratch holds 12 sigma
  const long long p0 = pidx(g, rhs, 0, x, y, 0);
  leapfrog_update<T, MODE, FORCED>(f, p0, f.u_cur[p0], ku * irh, s);
  leapfrog_update<T, MODE, FORCED>(f, p0 + g.field, f.u_cur[p0 + g.field], kv * irh, s);
}

template <typename T, int MODE, bool FORCED, int TL_TX, int TL_TY>
__global__ void __launch_bounds__(TL_TX * TL_TY) sbp_div2d_tl(Geom g, WaveFields<T> f, StepScalars s) {
  if (g.dim != 2) return;
  constexpr int SX = TL_TX + 2 * TL_H, SY = TL_TY + 2 * TL_H;
  __shared__ T sxx[TL_TY][SX];   // x-halo only
  __shared__ T syy[SY][TL_TX];   // y-halo only
  __shared__ T sxy[SY][SX];      // both
  const int rhs = blockIdx.z;
  const int x0 = blockIdx.x * TL_TX, y0 = blockIdx.y * TL_TY;
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
  if (!tl_block_interior<TL_TX, TL_TY>(g, x0, y0)) {
    pdl_wait();
    pdl_trigger();
    div2d_node<T, MODE, FORCED>(g, f, s, rhs, x, y);
    return;
  }
  const long long pc = pidx(g, 0, 0, x, y, 0);
  const long long p0 = pidx(g, rhs, 0, x, y, 0);
  const T irh = f.irh2[pc];                       // static: read before the wait
  pdl_wait();
  pdl_trigger();
  const T* base = f.sigma + (long long)rhs * 3 * g.field;
  const T* Gxx = base + pidx(g, 0, 0, x0 - TL_H, y0, 0);
  const T* Gyy = base + g.field + pidx(g, 0, 0, x0, y0 - TL_H, 0);
  const T* Gxy = base + 2 * g.field + pidx(g, 0, 0, x0 - TL_H, y0 - TL_H, 0);
  const int tid = threadIdx.y * TL_TX + threadIdx.x;
  for (int i = tid; i < SX * SY; i += TL_TX * TL_TY) {
    const int lx = i % SX, ly = i / SX;
    sxy[ly][lx] = Gxy[(long long)ly * g.np[0] + lx];
    if (ly < TL_TY) sxx[ly][lx] = Gxx[(long long)ly * g.np[0] + lx];
    if (lx < TL_TX) syy[ly][lx] = Gyy[(long long)ly * g.np[0] + lx];
  }
  const T u0 = f.u_cur[p0], u1 = f.u_cur[p0 + g.field];
  __syncthreads();
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int cx = tx + TL_H, cy = ty + TL_H;
  // 144 D sigma from 12 sigma
  const T ku = -c4u(sxx[ty][cx - 2], sxx[ty][cx - 1], sxx[ty][cx + 1], sxx[ty][cx + 2]) -
               c4u(sxy[cy - 2][cx], sxy[cy - 1][cx], sxy[cy + 1][cx], sxy[cy + 2][cx]);
  const T kv = -c4u(sxy[cy][cx - 2], sxy[cy][cx - 1], sxy[cy][cx + 1], sxy[cy][cx + 2]) -
               c4u(syy[cy - 2][tx], syy[cy - 1][tx], syy[cy + 1][tx], syy[cy + 2][tx]);
  const T irs = irh * T(1.0 / 144.0);
  leapfrog_update<T, MODE, FORCED>(f, p0, u0, ku * irs, s);
  leapfrog_update<T, MODE, FORCED>(f, p0 + g.field, u1, kv * irs, s);
}

// ---------------------------------------------------------------------------
// Order 4 (SBP), 2D, fused: one launch per time level.  A 32 x 16 tile (32 x 8
// in FP64, to stay within 48 KB of static shared memory) stages
// u on tile +- 6 nodes and lambda, mu on tile +- 3 in shared memory, forms the
// stresses on tile +- 3 (the closure rows reach 3 nodes), then the divergence
// and the leapfrog/filter update of its own nodes.
// ---------------------------------------------------------------------------
template <typename T>
__host__ __device__ constexpr int o4_tile_y() { return sizeof(T) == 8 ? 8 : 16; }

template <typename T, int MODE, bool FORCED>
__global__ void __launch_bounds__(512) step2d_o4_fused(Geom g, WaveFields<T> f, StepScalars s) {
  if (g.dim != 2) return;
  pdl_wait();
  pdl_trigger();
  constexpr int TX = 32, TY = o4_tile_y<T>(), HU = 6, HS = 3;
  constexpr int UX = TX + 2 * HU, UY = TY + 2 * HU;
  constexpr int SX = TX + 2 * HS, SY = TY + 2 * HS;
  __shared__ T su[2][UY][UX];
  __shared__ T sl[SY][SX];
  __shared__ T sm[SY][SX];
  __shared__ T ss[3][SY][SX];  // xx, yy, xy
  const int rhs = blockIdx.z;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int nx = g.n[0], ny = g.n[1];
  for (int i = tid; i < UX * UY; i += TX * TY) {
    const int lx = i % UX, ly = i / UX;
    const long long pu = pidx(g, rhs, 0, x0 - HU + lx, y0 - HU + ly, 0);
    su[0][ly][lx] = f.u_cur[pu];
    su[1][ly][lx] = f.u_cur[pu + g.field];
  }
  for (int i = tid; i < SX * SY; i += TX * TY) {
    const int lx = i % SX, ly = i / SX;
    const long long pc = pidx(g, 0, 0, x0 - HS + lx, y0 - HS + ly, 0);
    sl[ly][lx] = f.lam[pc];
    sm[ly][lx] = f.mu[pc];
  }
  __syncthreads();
  // stresses on the tile +- HS (nodes of the full grid only)
  for (int i = tid; i < SX * SY; i += TX * TY) {
    const int lx = i % SX, ly = i / SX;
    const int qx = x0 - HS + lx, qy = y0 - HS + ly;
    T sxx = T(0), syy = T(0), sxy = T(0);
    if (qx >= 0 && qx < nx && qy >= 0 && qy < ny) {
      const int ux = lx + (HU - HS), uy = ly + (HU - HS);
      const T u_x = sbp_d1<T>(&su[0][uy][ux], 1, qx, nx);
      const T u_y = sbp_d1<T>(&su[0][uy][ux], UX, qy, ny);
      const T v_x = sbp_d1<T>(&su[1][uy][ux], 1, qx, nx);
      const T v_y = sbp_d1<T>(&su[1][uy][ux], UX, qy, ny);
      const T l = sl[ly][lx], m = sm[ly][lx];
      const T div = u_x + v_y;
      sxx = l * div + T(2) * m * u_x;
      syy = l * div + T(2) * m * v_y;
      sxy = m * (u_y + v_x);
    }
    ss[0][ly][lx] = sxx;
    ss[1][ly][lx] = syy;
    ss[2][ly][lx] = sxy;
  }
  __syncthreads();
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
  if (!is_unknown(g, x, y, 0)) return;
  const int lx = threadIdx.x + HS, ly = threadIdx.y + HS;
  const T inv_h0 = T(48.0 / 17.0);
  // K u_x = -D_x sxx - D_y sxy (+ boundary terms on free sides)
  T ku = -sbp_d1<T>(&ss[0][ly][lx], 1, x, nx) - sbp_d1<T>(&ss[2][ly][lx], SX, y, ny);
  T kv = -sbp_d1<T>(&ss[2][ly][lx], 1, x, nx) - sbp_d1<T>(&ss[1][ly][lx], SX, y, ny);
  if (x == 0) {
    ku -= inv_h0 * ss[0][ly][lx];
    kv -= inv_h0 * ss[2][ly][lx];
  } else if (x == nx - 1) {
    ku += inv_h0 * ss[0][ly][lx];
    kv += inv_h0 * ss[2][ly][lx];
  }
  if (y == 0) {
    ku -= inv_h0 * ss[2][ly][lx];
    kv -= inv_h0 * ss[1][ly][lx];
  } else if (y == ny - 1) {
    ku += inv_h0 * ss[2][ly][lx];
    kv += inv_h0 * ss[1][ly][lx];
  }
  const T irh = f.irh2[pidx(g, 0, 0, x, y, 0)];
  const long long p0 = pidx(g, rhs, 0, x, y, 0);
  leapfrog_update<T, MODE, FORCED>(f, p0, su[0][threadIdx.y + HU][threadIdx.x + HU], ku * irh, s);
  leapfrog_update<T, MODE, FORCED>(f, p0 + g.field, su[1][threadIdx.y + HU][threadIdx.x + HU], kv * irh, s);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
// Launch with programmatic stream serialization (see pdl_wait); EWH_PDL=0
// turns it off.
static bool pdl_enabled() {
  const char* e = getenv("EWH_PDL");
  return !(e && e[0] == '0');
}

template <typename... KArgs, typename... Args>
static cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// 2D order-4 kernel variants (Geom::variant, chosen per context by the
// autotuner): 0..3 = stress + divergence launches with 32x8, 32x16, 64x8 or
// 64x4 blocks, 4 = single fused launch, YM_VARIANT = the FP32 y-march
// (ewh_ymarch.cu).  EWH_STEP2D_O4=fused|split|ym overrides it (read whenever
// launches are enqueued; a context captures its step graph once, on first use).
// Mapped 2D grids: 0 = fused curv_step2d with 32x8 outputs per block, 1 =
// curv_stress2d + curv_div2d, 2 = fused with 32x16 outputs (FP32; FP64 runs 32x8).  Geom::variant
// from the autotuner; EWH_CURV=fused|fused16|split overrides it.
static int curv_variant(const Geom& g) {
  const char* e = getenv("EWH_CURV");
  if (e && e[0] == 'f') return strcmp(e, "fused16") == 0 ? 2 : 0;
  if (e && e[0] == 's') return 1;
  return (g.variant == 1 || g.variant == 2) ? g.variant : 0;
}

static int step2d_o4_variant(const Geom& g) {
  const char* e = getenv("EWH_STEP2D_O4");
  if (e && e[0] == 'f') return 1;
  if (e && e[0] == 's') return 0;
  return g.variant == 4 ? 1 : 0;
}
static int step2d_o4_tile(const Geom& g) {
  const char* e = getenv("EWH_STEP2D_O4");
  if (e && e[0] == 's') return 0;
  return (g.variant >= 0 && g.variant <= 3) ? g.variant : 0;
}

// ---------------------------------------------------------------------------
// Order 4 (SBP), 2D, curvilinear grid (Section 4.1, curvilinear form): the
// node grid is the image of (q, r) = (i h, j h) under a smooth mapping.  The
// stress kernel forms physical derivatives from the SBP derivatives in q and
// r, u_x = (y_r u_q - y_q u_r) / J, u_y = (x_q u_r - x_r u_q) / J, the
// stresses (the 1/J rides on lambda / J and mu / J, which the context stores
// in place of lambda and mu), and the four J-weighted fluxes
//   F^q_u = y_r s_xx - x_r s_xy,  F^r_u = -y_q s_xx + x_q s_xy,
//   F^q_v = y_r s_xy - x_r s_yy,  F^r_v = -y_q s_xy + x_q s_yy;
// the divergence kernel forms -D_q F^q - D_r F^r + H^{-1} B F (the Cartesian
// kernel with the fluxes in place of the stresses) times 1/(rho J h^2).
// One node per thread, global memory (the grid sizes of mapped problems are
// moderate); the metric planes are (y_r, -x_r, -y_q, x_q).
// ---------------------------------------------------------------------------
// The block's nodes and their 2-node reach lie in rows and columns 4 .. n - 5
// (every difference central, every node an unknown): uniform per block.
__device__ __forceinline__ bool curv_block_inner(const Geom& g) {
  const int x0 = blockIdx.x * blockDim.x, y0 = blockIdx.y * blockDim.y;
  return x0 >= 4 && x0 + (int)blockDim.x - 1 <= g.n[0] - 5 && y0 >= 4 && y0 + (int)blockDim.y - 1 <= g.n[1] - 5;
}

template <typename T>
__global__ void __launch_bounds__(256) curv_stress2d(Geom g, const T* __restrict__ u, const T* __restrict__ lam,
                                                     const T* __restrict__ mu, const T* __restrict__ met,
                                                     T* __restrict__ sig) {
  if (g.dim != 2) return;
  pdl_wait();
  pdl_trigger();
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  const int rhs = blockIdx.z;
  if (x >= g.n[0] || y >= g.n[1]) return;
  const long long sy = g.np[0];
  const long long pc = pidx(g, 0, 0, x, y, 0);
  const T* U = u + pidx(g, rhs, 0, x, y, 0);
  const T* V = U + g.field;
  T uq, ur, vq, vr;
  if (curv_block_inner(g)) {  // central differences, 32-bit offsets
    const int s1 = g.np[0];
    uq = c4(U[-2], U[-1], U[1], U[2]);
    vq = c4(V[-2], V[-1], V[1], V[2]);
    ur = c4(U[-2 * s1], U[-s1], U[s1], U[2 * s1]);
    vr = c4(V[-2 * s1], V[-s1], V[s1], V[2 * s1]);
  } else {
    uq = sbp_d1<T>(U, 1, x, g.n[0]);
    ur = sbp_d1<T>(U, sy, y, g.n[1]);
    vq = sbp_d1<T>(V, 1, x, g.n[0]);
    vr = sbp_d1<T>(V, sy, y, g.n[1]);
  }
  const T a0 = met[pc], a1 = met[g.field + pc], a2 = met[2 * g.field + pc], a3 = met[3 * g.field + pc];
  const T u_x = a0 * uq + a2 * ur, u_y = a1 * uq + a3 * ur;  // J times the physical gradient
  const T v_x = a0 * vq + a2 * vr, v_y = a1 * vq + a3 * vr;
  const T l = lam[pc], m = mu[pc];                            // lambda / J, mu / J
  const T div = u_x + v_y;
  const T sxx = l * div + T(2) * m * u_x, syy = l * div + T(2) * m * v_y, sxy = m * (u_y + v_x);
  T* out = sig + (long long)rhs * 4 * g.field + pc;
  out[0] = a0 * sxx + a1 * sxy;
  out[g.field] = a2 * sxx + a3 * sxy;
  out[2 * g.field] = a0 * sxy + a1 * syy;
  out[3 * g.field] = a2 * sxy + a3 * syy;
}

template <typename T, int MODE, bool FORCED>
__global__ void __launch_bounds__(256) curv_div2d(Geom g, WaveFields<T> f, StepScalars s) {
  if (g.dim != 2) return;
  pdl_wait();
  pdl_trigger();
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  const int rhs = blockIdx.z;
  if (!is_unknown(g, x, y, 0)) return;
  const long long sy = g.np[0];
  const long long pc = pidx(g, 0, 0, x, y, 0);
  const T* fqu = f.sigma + (long long)rhs * 4 * g.field + pc;
  const T* fru = fqu + g.field;
  const T* fqv = fqu + 2 * g.field;
  const T* frv = fqu + 3 * g.field;
  if (curv_block_inner(g)) {  // central differences, no boundary terms
    const int s1 = g.np[0];
    const T ku = -c4(fqu[-2], fqu[-1], fqu[1], fqu[2]) - c4(fru[-2 * s1], fru[-s1], fru[s1], fru[2 * s1]);
    const T kv = -c4(fqv[-2], fqv[-1], fqv[1], fqv[2]) - c4(frv[-2 * s1], frv[-s1], frv[s1], frv[2 * s1]);
    const T irh = f.irh2[pc];
    const long long p0 = pidx(g, rhs, 0, x, y, 0);
    leapfrog_update<T, MODE, FORCED>(f, p0, f.u_cur[p0], ku * irh, s);
    leapfrog_update<T, MODE, FORCED>(f, p0 + g.field, f.u_cur[p0 + g.field], kv * irh, s);
    return;
  }
  T ku = -sbp_d1<T>(fqu, 1, x, g.n[0]) - sbp_d1<T>(fru, sy, y, g.n[1]);
  T kv = -sbp_d1<T>(fqv, 1, x, g.n[0]) - sbp_d1<T>(frv, sy, y, g.n[1]);
  const T inv_h0 = T(48.0 / 17.0);
  if (x == 0) {
    ku -= inv_h0 * fqu[0];
    kv -= inv_h0 * fqv[0];
  } else if (x == g.n[0] - 1) {
    ku += inv_h0 * fqu[0];
    kv += inv_h0 * fqv[0];
  }
  if (y == 0) {
    ku -= inv_h0 * fru[0];
    kv -= inv_h0 * frv[0];
  } else if (y == g.n[1] - 1) {
    ku += inv_h0 * fru[0];
    kv += inv_h0 * frv[0];
  }
  const T irh = f.irh2[pc];  // 1 / (rho J h^2)
  const long long p0 = pidx(g, rhs, 0, x, y, 0);
  leapfrog_update<T, MODE, FORCED>(f, p0, f.u_cur[p0], ku * irh, s);
  leapfrog_update<T, MODE, FORCED>(f, p0 + g.field, f.u_cur[p0 + g.field], kv * irh, s);
}

// Fused form of the two kernels above: one launch per time level, blocks of
// 32 x 8 threads and 32 x (8 RPT) output nodes (RPT rows per thread).  The
// block stages u (both components) and the six coefficient planes (y_r, -x_r,
// -y_q, x_q, lambda / J, mu / J) on a tile of (32 + 6) x (8 RPT + 6) nodes in
// shared memory, then forms the four fluxes in place of the first four
// planes.  The tile starts 2 nodes before the block, or at n - 6 when that is
// lower, so it holds every flux a central or SBP-closure difference of the
// block's nodes reads.  Blocks whose tile lies in rows and columns 4 .. n - 5
// (every difference central, every node an unknown) take a path with no
// per-node tests; the others difference fluxes at nodes within 4 of a side
// with the SBP closure applied to u in global memory.  Every load is issued
// before the first barrier: the coefficients (static) ahead of the wait on the
// previous level, the state and the update's operands after it.
template <typename T, int MODE, bool FORCED, int RPT>
__global__ void __launch_bounds__(256) curv_step2d(Geom g, WaveFields<T> f, StepScalars s) {
  if (g.dim != 2) return;
  constexpr int TX = 32, TY = 8 * RPT;
  constexpr int FX = TX + 6, FY = TY + 6;  // flux / coefficient tile
  constexpr int UX = FX + 4, UY = FY + 4;  // u tile: 2-node reach of the central fluxes
  __shared__ T su[2][UY][UX];
  __shared__ T sc[6][FY][FX];
  const int nx = g.n[0], ny = g.n[1];
  const int rhs = blockIdx.z;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int xs = min(x0 - 2, nx - 6), ys = min(y0 - 2, ny - 6);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int sy = g.np[0];
  const int fld = (int)g.field;  // one padded component indexes in 32 bits
  const bool inner = xs >= 4 && xs + FX - 1 <= nx - 5 && ys >= 4 && ys + FY - 1 <= ny - 5;
  const long long cbase = pidx(g, 0, 0, xs, ys, 0);  // coefficient tile origin
  const T* M0 = f.met + cbase;
  const T* LA = f.lam + cbase;
  const T* MU = f.mu + cbase;
  if (inner) {
    for (int r = ty; r < FY; r += 8)
      for (int c = tx; c < FX; c += 32) {
        const int q = r * sy + c;
        sc[0][r][c] = M0[q];
        sc[1][r][c] = M0[fld + q];
        sc[2][r][c] = M0[2 * fld + q];
        sc[3][r][c] = M0[3 * fld + q];
        sc[4][r][c] = LA[q];
        sc[5][r][c] = MU[q];
      }
  } else {
    for (int r = ty; r < FY; r += 8)
      for (int c = tx; c < FX; c += 32) {
        const int gx = xs + c, gy = ys + r;
        const bool in = gx >= 0 && gx < nx && gy >= 0 && gy < ny;
        const int q = r * sy + c;
        sc[0][r][c] = in ? M0[q] : T(0);
        sc[1][r][c] = in ? M0[fld + q] : T(0);
        sc[2][r][c] = in ? M0[2 * fld + q] : T(0);
        sc[3][r][c] = in ? M0[3 * fld + q] : T(0);
        sc[4][r][c] = in ? LA[q] : T(0);
        sc[5][r][c] = in ? MU[q] : T(0);
      }
  }
  // this thread's output nodes: (x0 + tx, y0 + ty + 8 k)
  const int x = x0 + tx;
  const long long p00 = pidx(g, rhs, 0, x, y0 + ty, 0);
  const long long c00 = pidx(g, 0, 0, x, y0 + ty, 0);
  bool unk[RPT];
  T irh[RPT], fr0[RPT], fr1[RPT];
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    unk[k] = inner || is_unknown(g, x, y0 + ty + 8 * k, 0);
    irh[k] = unk[k] ? f.irh2[c00 + 8 * k * sy] : T(0);  // 1 / (rho J h^2)
    fr0[k] = (FORCED && unk[k]) ? f.frho[p00 + 8 * k * sy] : T(0);
    fr1[k] = (FORCED && unk[k]) ? f.frho[p00 + 8 * k * sy + fld] : T(0);
  }
  pdl_wait();
  pdl_trigger();
  const T* U0 = f.u_cur + pidx(g, rhs, 0, 0, 0, 0);
  {
    const T* Ut = f.u_cur + pidx(g, rhs, 0, xs - 2, ys - 2, 0);  // inside the padding (PAD >= 4)
    for (int r = ty; r < UY; r += 8)
      for (int c = tx; c < UX; c += 32) {
        const int gx = xs - 2 + c, gy = ys - 2 + r;
        const bool in = inner || (gx >= 0 && gx < nx && gy >= 0 && gy < ny);
        const int q = r * sy + c;
        su[0][r][c] = in ? Ut[q] : T(0);
        su[1][r][c] = in ? Ut[fld + q] : T(0);
      }
  }
  T d0[RPT], d1[RPT], ac0[RPT], ac1[RPT];
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const bool ld = MODE != 3 && MODE != STEP_FIRST && unk[k];
    const long long p = p00 + 8 * k * sy;
    d0[k] = ld ? f.delta[p] : T(0);
    d1[k] = ld ? f.delta[p + fld] : T(0);
    ac0[k] = ld ? f.acc[p] : T(0);
    ac1[k] = ld ? f.acc[p + fld] : T(0);
  }
  __syncthreads();
  for (int r = ty; r < FY; r += 8)
    for (int c = tx; c < FX; c += 32) {
      const int gx = xs + c, gy = ys + r;
      T uq, ur, vq, vr;
      const int ux = c + 2, uy = r + 2;
      if (inner || (gx >= 4 && gx <= nx - 5)) {
        uq = c4(su[0][uy][ux - 2], su[0][uy][ux - 1], su[0][uy][ux + 1], su[0][uy][ux + 2]);
        vq = c4(su[1][uy][ux - 2], su[1][uy][ux - 1], su[1][uy][ux + 1], su[1][uy][ux + 2]);
      } else {
        if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) continue;  // never read
        const long long q = (long long)gy * sy + gx;
        uq = sbp_d1<T>(U0 + q, 1, gx, nx);
        vq = sbp_d1<T>(U0 + fld + q, 1, gx, nx);
      }
      if (inner || (gy >= 4 && gy <= ny - 5)) {
        ur = c4(su[0][uy - 2][ux], su[0][uy - 1][ux], su[0][uy + 1][ux], su[0][uy + 2][ux]);
        vr = c4(su[1][uy - 2][ux], su[1][uy - 1][ux], su[1][uy + 1][ux], su[1][uy + 2][ux]);
      } else {
        if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) continue;  // never read
        const long long q = (long long)gy * sy + gx;
        ur = sbp_d1<T>(U0 + q, sy, gy, ny);
        vr = sbp_d1<T>(U0 + fld + q, sy, gy, ny);
      }
      const T a0 = sc[0][r][c], a1 = sc[1][r][c], a2 = sc[2][r][c], a3 = sc[3][r][c];
      const T l = sc[4][r][c], m = sc[5][r][c];
      const T u_x = a0 * uq + a2 * ur, u_y = a1 * uq + a3 * ur;
      const T v_x = a0 * vq + a2 * vr, v_y = a1 * vq + a3 * vr;
      const T div = u_x + v_y;
      const T sxx = l * div + T(2) * m * u_x, syy = l * div + T(2) * m * v_y, sxy = m * (u_y + v_x);
      sc[0][r][c] = a0 * sxx + a1 * sxy;
      sc[1][r][c] = a2 * sxx + a3 * sxy;
      sc[2][r][c] = a0 * sxy + a1 * syy;
      sc[3][r][c] = a2 * sxy + a3 * syy;
    }
  __syncthreads();
  const int lx = x - xs;
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    if (!unk[k]) continue;
    const int y = y0 + ty + 8 * k;
    const int ly = y - ys;
    const T* fqu = &sc[0][ly][lx];
    const T* fru = &sc[1][ly][lx];
    const T* fqv = &sc[2][ly][lx];
    const T* frv = &sc[3][ly][lx];
    T ku, kv;
    if (inner || (x >= 4 && x <= nx - 5)) {
      ku = -c4(fqu[-2], fqu[-1], fqu[1], fqu[2]);
      kv = -c4(fqv[-2], fqv[-1], fqv[1], fqv[2]);
    } else {
      ku = -sbp_d1<T>(fqu, 1, x, nx);
      kv = -sbp_d1<T>(fqv, 1, x, nx);
    }
    if (inner || (y >= 4 && y <= ny - 5)) {
      ku -= c4(fru[-2 * FX], fru[-FX], fru[FX], fru[2 * FX]);
      kv -= c4(frv[-2 * FX], frv[-FX], frv[FX], frv[2 * FX]);
    } else {
      ku -= sbp_d1<T>(fru, FX, y, ny);
      kv -= sbp_d1<T>(frv, FX, y, ny);
    }
    if (!inner) {
      const T inv_h0 = T(48.0 / 17.0);
      if (x == 0) {
        ku -= inv_h0 * fqu[0];
        kv -= inv_h0 * fqv[0];
      } else if (x == nx - 1) {
        ku += inv_h0 * fqu[0];
        kv += inv_h0 * fqv[0];
      }
      if (y == 0) {
        ku -= inv_h0 * fru[0];
        kv -= inv_h0 * frv[0];
      } else if (y == ny - 1) {
        ku += inv_h0 * fru[0];
        kv += inv_h0 * frv[0];
      }
    }
    const long long p = p00 + 8 * k * sy;
    leapfrog_update_pre<T, MODE, FORCED>(f, p, su[0][ly + 2][lx + 2], ku * irh[k], s, d0[k], ac0[k], fr0[k]);
    leapfrog_update_pre<T, MODE, FORCED>(f, p + fld, su[1][ly + 2][lx + 2], kv * irh[k], s, d1[k], ac1[k], fr1[k]);
  }
}

// Metric terms of a mapped grid (FP64, dense C-order planes, x fastest):
// x_q, x_r, y_q, y_r from the SBP first derivative over the node spacing h,
// J = x_q y_r - x_r y_q; out holds the planes (y_r, -x_r, -y_q, x_q, 1/J, J).
__global__ void curv_metrics_kernel(int n0, int n1, double h, const double* __restrict__ X,
                                    const double* __restrict__ Y, double* __restrict__ out) {
  const long long total = (long long)n0 * n1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % n0), y = (int)(i / n0);
    const double xq = sbp_d1<double>(X + i, 1, x, n0) / h, xr = sbp_d1<double>(X + i, n0, y, n1) / h;
    const double yq = sbp_d1<double>(Y + i, 1, x, n0) / h, yr = sbp_d1<double>(Y + i, n0, y, n1) / h;
    const double J = xq * yr - xr * yq;
    out[i] = yr;
    out[total + i] = -xr;
    out[2 * total + i] = -yq;
    out[3 * total + i] = xq;
    out[4 * total + i] = 1.0 / J;
    out[5 * total + i] = J;
  }
}

cudaError_t launch_curv_metrics(int n0, int n1, double h, const double* X, const double* Y, double* out,
                                cudaStream_t st) {
  const long long total = (long long)n0 * n1;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 4096);
  curv_metrics_kernel<<<blocks, 256, 0, st>>>(n0, n1, h, X, Y, out);
  return cudaGetLastError();
}

template <typename T, int MODE, bool FORCED, int TX, int TY>
static cudaError_t launch_split_o4(const Geom& g, const WaveFields<T>& f, const StepScalars& s, cudaStream_t st) {
  dim3 tgrd((g.n[0] + TX - 1) / TX, (g.n[1] + TY - 1) / TY, g.nrhs);
  cudaError_t e = launch_k(sbp_stress2d_tl<T, TX, TY>, tgrd, dim3(TX, TY), st, g, (const T*)f.u_cur, f.lam, f.mu,
                           f.sigma);
  if (e != cudaSuccess) return e;
  return launch_k(sbp_div2d_tl<T, MODE, FORCED, TX, TY>, tgrd, dim3(TX, TY), st, g, f, s);
}

template <typename T, int MODE, bool FORCED>
static cudaError_t launch_mode(const Geom& g, int order, const WaveFields<T>& f, const StepScalars& s,
                               cudaStream_t st, long long* nl) {
  if (order == 2) {
    if (g.dim == 2) {
      // tile height chosen per context (autotuner): 0 -> 8, 1 -> 4, 2 -> 16 rows
      const int ty = g.variant == 1 ? 4 : (g.variant == 2 ? 16 : 8);
      dim3 blk(32, ty), grd((g.n[0] + 31) / 32, (g.n[1] + ty - 1) / ty, g.nrhs);
      cudaError_t e = ty == 4    ? launch_k(step2d_o2<T, MODE, FORCED, 4>, grd, blk, st, g, f, s)
                      : ty == 16 ? launch_k(step2d_o2<T, MODE, FORCED, 16>, grd, blk, st, g, f, s)
                                 : launch_k(step2d_o2<T, MODE, FORCED, 8>, grd, blk, st, g, f, s);
      if (e != cudaSuccess) return e;
    } else {
      dim3 blk(32, 4, 2), grd((g.n[0] + 31) / 32, (g.n[1] + 3) / 4, ((g.n[2] + 1) / 2) * g.nrhs);
      cudaError_t e = launch_k(step3d_o2<T, MODE, FORCED>, grd, blk, st, g, f, s);
      if (e != cudaSuccess) return e;
    }
    if (nl) *nl += 1;
    return cudaGetLastError();
  }
  if (g.mapped) {  // curvilinear 2D order 4: fused 32x8 (0) or 32x16 (2, FP32), stress + divergence (1)
    const int cv = curv_variant(g);
    if (cv != 1) {
      cudaError_t e;
      if (cv == 2 && sizeof(T) == 4) {  // 32 x 16 outputs per block
        dim3 blk(32, 8), grd((g.n[0] + 31) / 32, (g.n[1] + 15) / 16, g.nrhs);
        e = launch_k(curv_step2d<T, MODE, FORCED, sizeof(T) == 4 ? 2 : 1>, grd, blk, st, g, f, s);
      } else {
        dim3 blk(32, 8), grd((g.n[0] + 31) / 32, (g.n[1] + 7) / 8, g.nrhs);
        e = launch_k(curv_step2d<T, MODE, FORCED, 1>, grd, blk, st, g, f, s);
      }
      if (e != cudaSuccess) return e;
      if (nl) *nl += 1;
      return cudaGetLastError();
    }
    dim3 blk(32, 8), grd((g.n[0] + 31) / 32, (g.n[1] + 7) / 8, g.nrhs);
    cudaError_t e = launch_k(curv_stress2d<T>, grd, blk, st, g, (const T*)f.u_cur, f.lam, f.mu, f.met, f.sigma);
    if (e != cudaSuccess) return e;
    e = launch_k(curv_div2d<T, MODE, FORCED>, grd, blk, st, g, f, s);
    if (e != cudaSuccess) return e;
    if (nl) *nl += 2;
    return cudaGetLastError();
  }
  if constexpr (sizeof(T) == 4 && MODE != 3) {
    // fused y-march: autotuner variant YM_VARIANT; EWH_STEP2D_O4=ym forces it
    const char* ev = getenv("EWH_STEP2D_O4");
    const bool ym = ev ? strcmp(ev, "ym") == 0 : g.variant == YM_VARIANT;
    if (g.dim == 2 && ym && f.zm && f.zm->ok[0]) {
      cudaError_t e = launch_ymarch(g, *f.zm, f, (StepMode)MODE, s, st);
      if (e != cudaSuccess) return e;
      if (nl) *nl += 1;
      return cudaGetLastError();
    }
  }
  if (g.dim == 2 && step2d_o4_variant(g) == 1) {
    constexpr int TY = o4_tile_y<T>();
    dim3 blk(32, TY), grd((g.n[0] + 31) / 32, (g.n[1] + TY - 1) / TY, g.nrhs);
    cudaError_t e = launch_k(step2d_o4_fused<T, MODE, FORCED>, grd, blk, st, g, f, s);
    if (e != cudaSuccess) return e;
    if (nl) *nl += 1;
    return cudaGetLastError();
  }
  dim3 blk(32, 8);
  dim3 grd((g.n[0] + 31) / 32, (g.n[1] + 7) / 8, g.dim == 2 ? g.nrhs : g.n[2] * g.nrhs);
  if (g.dim == 2) {
    const int tv = step2d_o4_tile(g);
    cudaError_t e = tv == 1   ? launch_split_o4<T, MODE, FORCED, 32, 16>(g, f, s, st)
                    : tv == 2 ? launch_split_o4<T, MODE, FORCED, 64, 8>(g, f, s, st)
                    : tv == 3 ? launch_split_o4<T, MODE, FORCED, 64, 4>(g, f, s, st)
                              : launch_split_o4<T, MODE, FORCED, 32, 8>(g, f, s, st);
    if (e != cudaSuccess) return e;
  } else {
    if constexpr (sizeof(T) == 4 && MODE != 3) {
      // fused z-march: autotuner variants 1 (32 x 16 tiles) and 2 (32 x 8);
      // EWH_STEP3D_O4=pair|zm16|zm8 (zm: 32 x 8) overrides it
      const char* ev = getenv("EWH_STEP3D_O4");
      int zk = g.variant == 1 ? 0 : (g.variant == 2 ? 1 : -1);
      if (ev) zk = ev[0] != 'z' ? -1 : (strcmp(ev, "zm16") == 0 ? 0 : 1);
      if (zk >= 0 && f.zm && f.zm->ok[zk]) {
        cudaError_t e = launch_zmarch(g, *f.zm, zk, f, (StepMode)MODE, s, st);
        if (e != cudaSuccess) return e;
        if (nl) *nl += 1;
        return cudaGetLastError();
      }
    }
    cudaError_t e = launch_k(sbp_stress<T, 3>, grd, blk, st, g, (const T*)f.u_cur, f.lam, f.mu, f.sigma);
    if (e != cudaSuccess) return e;
    e = launch_k(sbp_divergence_step<T, 3, MODE, FORCED>, grd, blk, st, g, f, s);
    if (e != cudaSuccess) return e;
  }
  if (nl) *nl += 2;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_step(const Geom& g, int order, const WaveFields<T>& f, StepMode mode,
                        const StepScalars& s, cudaStream_t st, long long* nl) {
  const bool forced = f.frho != nullptr;
  switch (mode) {
    case STEP_FIRST:
      return forced ? launch_mode<T, STEP_FIRST, true>(g, order, f, s, st, nl)
                    : launch_mode<T, STEP_FIRST, false>(g, order, f, s, st, nl);
    case STEP_MID:
      return forced ? launch_mode<T, STEP_MID, true>(g, order, f, s, st, nl)
                    : launch_mode<T, STEP_MID, false>(g, order, f, s, st, nl);
    default:
      return forced ? launch_mode<T, STEP_LAST, true>(g, order, f, s, st, nl)
                    : launch_mode<T, STEP_LAST, false>(g, order, f, s, st, nl);
  }
}

template <typename T>
cudaError_t launch_minvK(const Geom& g, int order, const T* u, T* out, const T* lam, const T* mu,
                         const T* irh2, T* sigma, cudaStream_t st, long long* nl, const T* met) {
  WaveFields<T> f{};
  f.met = met;
  f.u_cur = const_cast<T*>(u);
  f.u_next = out;
  f.lam = lam;
  f.mu = mu;
  f.irh2 = irh2;
  f.frho = nullptr;
  f.sigma = sigma;
  StepScalars s{};
  return launch_mode<T, 3, false>(g, order, f, s, st, nl);
}

// ---------------------------------------------------------------------------
// Order 4 (SBP), 2D, FP32: every time level of a wave solve in ONE
// cooperative launch per group of right-hand sides, with the state held on
// chip.
//
// One CTA of NT threads per SM owns a wx x wy block of nodes of one
// right-hand side (every block at least 8 x 8, so SBP closure reaches stay
// inside the halos); a launch holds px x py blocks of each of rg right-hand
// sides, and the groups of a multi-rhs context run one launch after another.  Its nodes
// on central rows and columns (x, y in [4, n - 5]) form a rectangle, done in
// pairs along x with no per-node test; the others (within 4 nodes of a side:
// SBP closures, boundary terms, Dirichlet nodes) are special and take a pass
// of their own with the general code.  The CTA keeps
//   in shared memory: u on the block +- 4 nodes, the stresses on the block
//                     +- 2 nodes, delta on the block, the special nodes'
//                     filter accumulators;
//   in registers:     the filter accumulators of its regular node pairs
//                     (pair t + NT k of the rectangle for thread t, k < NP).
// Per time level a CTA reloads only the 4-node halo ring of u (its
// neighbours' rims, written at the previous level to a global exchange
// buffer), recomputes the stresses on block +- 2 from u on block +- 4, forms
// -D sigma + H^{-1} B sigma and the leapfrog/filter update of its own nodes
// (same arithmetic as the split kernels), writes its own 4-node rim to the
// other exchange buffer and counts itself in at a grid barrier; the central
// stresses of the next level that need no halo are computed before it waits
// there.  One barrier per level; lambda, mu, 1/(rho h^2) (and f/rho) are the
// only other global reads.  Barrier waits are bounded in time; on a timeout
// the kernel raises an error flag, every CTA leaves at its next barrier and
// fills its accumulator nodes with NaN, which the solve reports as a
// breakdown.
// ---------------------------------------------------------------------------
constexpr int RS_HU = 4;  // u halo
constexpr int RS_HS = 2;  // stress halo

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier pieces: a release add to count a CTA in, acquire loads to
// poll (see rs_arrive / rs_wait).
__device__ __forceinline__ void red_release_gpu(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}


// Split form of the grid barrier: rs_arrive after a __syncthreads that
// orders the CTA's writes (thread 0 counts the CTA in with a release add);
// rs_wait polls until `target` CTAs have arrived (each wait bounded: it gives
// up after `lim` ns or 2^22 polls, or when another CTA raised the error flag,
// which it then sees every 256 polls; a zero limit gives up at once, without
// polling) and ends with a __syncthreads.  Work that needs none of the other
// CTAs' data goes between the two.
__device__ __forceinline__ void rs_arrive(unsigned* bar) {
  if (threadIdx.x == 0) red_release_gpu(bar, 1u);
}

// Raise the error flag; the CTA that raises it first counts the launch in
// bar[4].  Returns 0 (the wait failed).
__device__ __forceinline__ int rs_give_up(unsigned* bar) {
  if (atomicExch(bar + 1, 1u) == 0u) atomicAdd(bar + 4, 1u);
  return 0;
}

__device__ __forceinline__ bool rs_wait(unsigned* bar, unsigned target, int* s_ok, unsigned long long lim) {
  if (threadIdx.x == 0) {
    int ok = ld_acquire_gpu(bar + 1) == 0u;
    if (ok && lim == 0ull) ok = rs_give_up(bar);
    const unsigned long long t0 = global_ns();
    for (unsigned spins = 1; ok && ld_acquire_gpu(bar) < target; ++spins) {
      if ((spins & 255u) == 0u) {
        if (ld_acquire_gpu(bar + 1) != 0u) {
          ok = 0;
        } else if (spins > (1u << 22) || global_ns() - t0 > lim) {
          ok = rs_give_up(bar);
        }
      }
    }
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

__device__ __forceinline__ bool rs_closure(int x, int n) { return x < 4 || x > n - 5; }

struct ResidentShape {
  int px, bx, by, ex;  // CTAs along x; interior block width; block height; first block width
  int nb;              // CTAs per right-hand side (px * py): CTA b holds block b % nb of rhs b / nb
};

// The shared-memory layout is fixed at compile time (so every stencil and
// plane offset is an immediate): blocks are at most RS_BXMAX x RS_BYMAX nodes.
constexpr int RS_BXMAX = 132;
constexpr int RS_BYMAX = 54;
constexpr int RS_UX = RS_BXMAX + 2 * RS_HU;  // u tile row stride
constexpr int RS_SX = RS_BXMAX + 2 * RS_HS;  // stress tile row stride
constexpr int RS_UPLANE = (RS_BYMAX + 2 * RS_HU) * RS_UX;
constexpr int RS_SPLANE = (RS_BYMAX + 2 * RS_HS) * RS_SX;
constexpr int RS_DPLANE = RS_BYMAX * RS_BXMAX;
constexpr int RS_OFF_V = RS_UPLANE;              // u, component 1
constexpr int RS_OFF_XX = 2 * RS_UPLANE;         // stresses xx, yy, xy
constexpr int RS_OFF_YY = RS_OFF_XX + RS_SPLANE;
constexpr int RS_OFF_XY = RS_OFF_YY + RS_SPLANE;
constexpr int RS_OFF_DU = RS_OFF_XY + RS_SPLANE;  // delta, components 0 and 1
constexpr int RS_OFF_DV = RS_OFF_DU + RS_DPLANE;
constexpr int RS_OFF_TAB = RS_OFF_DV + RS_DPLANE;  // copy of the SBP closure rows (4 x 6)
extern __shared__ float rs_smem[];  // dynamic shared memory of the resident kernel

// Own nodes on an SBP closure row or column (within 4 nodes of a side of the
// grid) are updated in a pass of their own; their filter accumulators live
// here (2 per node, at most RS_SPECIAL_MAX nodes per block).
constexpr int RS_SPECIAL_MAX = 1400;
constexpr int RS_OFF_SACC = RS_OFF_TAB + 24;
constexpr int RS_FLOATS = RS_OFF_SACC + 2 * RS_SPECIAL_MAX;

// Position j of the part of a W x H region outside the rectangle
// [x0, x1) x [y0, y1) (which may be empty: then y0 = H): rows [0, y0), rows
// [y1, H), then columns [0, x0) and [x1, W) of the rows between.  It has
// W H - (x1 - x0)(y1 - y0) positions.
__device__ __forceinline__ void rs_frame_pos(int j, int W, int H, int x0, int x1, int y0, int y1, int& x, int& y) {
  const int top = y0 * W;
  if (j < top) {
    y = j / W;
    x = j - y * W;
    return;
  }
  j -= top;
  const int bot = (H - y1) * W;
  if (j < bot) {
    const int r = j / W;
    y = y1 + r;
    x = j - r * W;
    return;
  }
  j -= bot;
  const int sw = x0 + (W - x1);
  const int r = j / sw, c = j - r * sw;
  y = y0 + r;
  x = c < x0 ? c : x1 + (c - x0);
}

// SBP first derivative as sbp_d1, with the closure rows read from the shared
// copy `tab`: lanes on different closure rows then read different banks
// instead of serialising on the constant cache.
__device__ __forceinline__ float rs_sbp_d1(const float* v, int s, int p, int N, const float* tab) {
  if (p < 4) {
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < 6; ++j) acc += tab[p * 6 + j] * v[(j - p) * s];
    return acc;
  }
  if (p > N - 5) {
    const int r = N - 1 - p;
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < 6; ++j) acc -= tab[r * 6 + j] * v[(r - j) * s];
    return acc;
  }
  return (v[-2 * s] - 8.0f * v[-s] + 8.0f * v[s] - v[2 * s]) * (1.0f / 12.0f);
}

// Advance a thread's position in a w-wide row-major walk by (sx, sy) = the
// thread count split into whole rows and a remainder.
__device__ __forceinline__ void walk_next(int& x, int& y, int w, int sx, int sy) {
  x += sx;
  y += sy;
  if (x >= w) {
    x -= w;
    ++y;
  }
}

// Stresses at one stress-tile position (qx, qy) of the block at (X0, Y0):
// the general form (SBP closures; nothing outside the grid).
__device__ __forceinline__ void rs_stress_gen(const float* __restrict__ lam, const float* __restrict__ mu, int n0,
                                              int n1, int npx, int X0, int Y0, int obase, int qx, int qy,
                                              const float* tab) {
  const int x = X0 + qx - RS_HS, y = Y0 + qy - RS_HS;
  if (x < 0 || x >= n0 || y < 0 || y >= n1) return;
  const int o = obase + (qy - RS_HS) * npx + (qx - RS_HS);
  const float l = __ldg(lam + o), m = __ldg(mu + o);
  const int pu = (qy + RS_HU - RS_HS) * RS_UX + (qx + RS_HU - RS_HS);
  const float* U = rs_smem + pu;
  const float* V = rs_smem + RS_OFF_V + pu;
  float u_x, v_x, u_y, v_y;
  if (x < 4 || x > n0 - 5) {
    u_x = rs_sbp_d1(U, 1, x, n0, tab);
    v_x = rs_sbp_d1(V, 1, x, n0, tab);
  } else {
    u_x = c4(U[-2], U[-1], U[1], U[2]);
    v_x = c4(V[-2], V[-1], V[1], V[2]);
  }
  if (y < 4 || y > n1 - 5) {
    u_y = rs_sbp_d1(U, RS_UX, y, n1, tab);
    v_y = rs_sbp_d1(V, RS_UX, y, n1, tab);
  } else {
    u_y = c4(U[-2 * RS_UX], U[-RS_UX], U[RS_UX], U[2 * RS_UX]);
    v_y = c4(V[-2 * RS_UX], V[-RS_UX], V[RS_UX], V[2 * RS_UX]);
  }
  const float div = u_x + v_y;
  const int ps = qy * RS_SX + qx;
  rs_smem[RS_OFF_XX + ps] = l * div + 2.0f * m * u_x;
  rs_smem[RS_OFF_YY + ps] = l * div + 2.0f * m * v_y;
  rs_smem[RS_OFF_XY + ps] = m * (u_y + v_x);
}

// Stresses at the central positions (qx, qy) and (qx + 1, qy), qx even,
// with 8-byte shared accesses (every plane offset and row stride is even).
__device__ __forceinline__ void rs_stress_pair(const float* __restrict__ lam, const float* __restrict__ mu, int npx,
                                               int obase, int qx, int qy) {
  const int o = obase + (qy - RS_HS) * npx + (qx - RS_HS);
  const float l0 = __ldg(lam + o), l1 = __ldg(lam + o + 1);
  const float m0 = __ldg(mu + o), m1 = __ldg(mu + o + 1);
  const int pu = (qy + RS_HU - RS_HS) * RS_UX + (qx + RS_HU - RS_HS);  // even
  const float2* U = reinterpret_cast<const float2*>(rs_smem + pu);
  const float2* V = reinterpret_cast<const float2*>(rs_smem + RS_OFF_V + pu);
  constexpr int RU = RS_UX / 2;
  const float2 ua = U[-1], ub = U[0], uc = U[1];
  const float2 va = V[-1], vb = V[0], vc = V[1];
  const float ux0 = c4(ua.x, ua.y, ub.y, uc.x), ux1 = c4(ua.y, ub.x, uc.x, uc.y);
  const float vx0 = c4(va.x, va.y, vb.y, vc.x), vx1 = c4(va.y, vb.x, vc.x, vc.y);
  const float2 um2 = U[-2 * RU], um1 = U[-RU], up1 = U[RU], up2 = U[2 * RU];
  const float2 vm2 = V[-2 * RU], vm1 = V[-RU], vp1 = V[RU], vp2 = V[2 * RU];
  const float uy0 = c4(um2.x, um1.x, up1.x, up2.x), uy1 = c4(um2.y, um1.y, up1.y, up2.y);
  const float vy0 = c4(vm2.x, vm1.x, vp1.x, vp2.x), vy1 = c4(vm2.y, vm1.y, vp1.y, vp2.y);
  const float div0 = ux0 + vy0, div1 = ux1 + vy1;
  const int ps = qy * RS_SX + qx;  // even
  *reinterpret_cast<float2*>(rs_smem + RS_OFF_XX + ps) =
      make_float2(l0 * div0 + 2.0f * m0 * ux0, l1 * div1 + 2.0f * m1 * ux1);
  *reinterpret_cast<float2*>(rs_smem + RS_OFF_YY + ps) =
      make_float2(l0 * div0 + 2.0f * m0 * vy0, l1 * div1 + 2.0f * m1 * vy1);
  *reinterpret_cast<float2*>(rs_smem + RS_OFF_XY + ps) = make_float2(m0 * (uy0 + vx0), m1 * (uy1 + vx1));
}

// Per-level scalars of the leapfrog/filter update.
struct RsLevel {
  float kt, w0, wnew, cosn;
  int first;  // level 0: Taylor start
  int last;   // last level: u^{n+1} is not stored
};

// -D sigma + H^{-1} B sigma at own node (ix, iy), times 1/(rho h^2), plus the
// forcing: the general form (SBP closures, boundary terms).
__device__ __forceinline__ void rs_accel_gen(const Geom& g, const float* __restrict__ irh2,
                                             const float* __restrict__ frho, int F, int X0, int Y0, int obase, int ix,
                                             int iy, const RsLevel& L, const float* tab, float& au, float& av) {
  const int n0 = g.n[0], n1 = g.n[1];
  const int x = X0 + ix, y = Y0 + iy;
  const int ps = (iy + RS_HS) * RS_SX + (ix + RS_HS);
  const float* Sxx = rs_smem + RS_OFF_XX + ps;
  const float* Syy = rs_smem + RS_OFF_YY + ps;
  const float* Sxy = rs_smem + RS_OFF_XY + ps;
  float kxu, kxv, kyu, kyv;
  if (x < 4 || x > n0 - 5) {
    kxu = rs_sbp_d1(Sxx, 1, x, n0, tab);
    kxv = rs_sbp_d1(Sxy, 1, x, n0, tab);
  } else {
    kxu = c4(Sxx[-2], Sxx[-1], Sxx[1], Sxx[2]);
    kxv = c4(Sxy[-2], Sxy[-1], Sxy[1], Sxy[2]);
  }
  if (y < 4 || y > n1 - 5) {
    kyu = rs_sbp_d1(Sxy, RS_SX, y, n1, tab);
    kyv = rs_sbp_d1(Syy, RS_SX, y, n1, tab);
  } else {
    kyu = c4(Sxy[-2 * RS_SX], Sxy[-RS_SX], Sxy[RS_SX], Sxy[2 * RS_SX]);
    kyv = c4(Syy[-2 * RS_SX], Syy[-RS_SX], Syy[RS_SX], Syy[2 * RS_SX]);
  }
  float ku = -kxu - kyu;
  float kv = -kxv - kyv;
  const float inv_h0 = 48.0f / 17.0f;
  if (x == 0) {
    ku -= inv_h0 * Sxx[0];
    kv -= inv_h0 * Sxy[0];
  } else if (x == n0 - 1) {
    ku += inv_h0 * Sxx[0];
    kv += inv_h0 * Sxy[0];
  }
  if (y == 0) {
    ku -= inv_h0 * Sxy[0];
    kv -= inv_h0 * Syy[0];
  } else if (y == n1 - 1) {
    ku += inv_h0 * Sxy[0];
    kv += inv_h0 * Syy[0];
  }
  const int o = obase + iy * g.np[0] + ix;
  const float irh = __ldg(irh2 + o);
  au = ku * irh;
  av = kv * irh;
  if (frho) {
    au += __ldg(frho + o) * L.cosn;
    av += __ldg(frho + F + o) * L.cosn;
  }
}

// Leapfrog/filter update of own node (ix, iy) from its accelerations (the
// arithmetic of leapfrog_update in FP32): delta and u in shared memory, the
// accumulators in acu, acv.
__device__ __forceinline__ void rs_update(int ix, int iy, float au, float av, const RsLevel& L, float& acu,
                                          float& acv) {
  const int pu = (iy + RS_HU) * RS_UX + (ix + RS_HU);
  const int pd = iy * RS_BXMAX + ix;
  const float uu = rs_smem[pu], uv = rs_smem[RS_OFF_V + pu];
  float du, dv;
  if (L.first) {
    du = -0.5f * L.kt * au;
    dv = -0.5f * L.kt * av;
  } else {
    du = rs_smem[RS_OFF_DU + pd] - L.kt * au;
    dv = rs_smem[RS_OFF_DV + pd] - L.kt * av;
  }
  const float nu_ = uu + du, nv_ = uv + dv;
  if (L.first) {
    acu = L.w0 * uu + L.wnew * nu_;
    acv = L.w0 * uv + L.wnew * nv_;
  } else {
    acu += L.wnew * nu_;
    acv += L.wnew * nv_;
  }
  rs_smem[RS_OFF_DU + pd] = du;
  rs_smem[RS_OFF_DV + pd] = dv;
  if (!L.last) {
    rs_smem[pu] = nu_;
    rs_smem[RS_OFF_V + pu] = nv_;
  }
}

template <int NT, int NP>
__global__ void __launch_bounds__(NT, 1) step2d_o4_resident(Geom g, ResidentShape sh, ResidentIO iop) {
  if (g.dim != 2) return;
  __shared__ int s_ok;
  const unsigned long long wait_ns = *reinterpret_cast<const unsigned long long*>(iop.bar + 2);
  const int n0 = g.n[0], n1 = g.n[1];
  // this CTA's right-hand side (of the launch's group) and block
  const int rloc = blockIdx.x / sh.nb, bid = blockIdx.x - rloc * sh.nb;
  ResidentIO io = iop;
  {
    const long long ro = (long long)rloc * 2 * g.field;
    io.u0 += ro;
    io.xbuf0 += ro;
    io.xbuf1 += ro;
    io.acc += ro;
    if (io.frho) io.frho += ro;
  }
  const int cx = bid % sh.px;
  const int X0 = cx == 0 ? 0 : sh.ex + (cx - 1) * sh.bx, Y0 = (bid / sh.px) * sh.by;
  const int wx = cx == 0 ? sh.ex : min(sh.bx, n0 - X0), wy = min(sh.by, n1 - Y0);
  // u: [RS_BYMAX + 8][RS_UX] per component, block node (0, 0) at (4, 4);
  // stresses: [RS_BYMAX + 4][RS_SX], block node (0, 0) at (2, 2);
  // delta of the own nodes: [RS_BYMAX][RS_BXMAX]
  float* const su = rs_smem;
  float* const sv = rs_smem + RS_OFF_V;
  float* const sxx = rs_smem + RS_OFF_XX;
  float* const syy = rs_smem + RS_OFF_YY;
  float* const sxy = rs_smem + RS_OFF_XY;
  float* const tab = rs_smem + RS_OFF_TAB;
  float* const sacc = rs_smem + RS_OFF_SACC;
  const int t = threadIdx.x;
  const int F = (int)g.field;  // < 2^31 (checked at creation)
  const int npx = g.np[0];
  const int obase = (Y0 + PAD) * npx + X0 + g.padx;     // padded offset of block node (0, 0)
  const int ubase = obase - RS_HU * npx - RS_HU;         // ... of u tile position (0, 0)
  const int ux = wx + 2 * RS_HU, uy = wy + 2 * RS_HU;
  const int sxn = wx + 2 * RS_HS, syn = wy + 2 * RS_HS;
  // Stress positions on central rows and columns (x and y in [4, n - 5]):
  // the rectangle [qa, qb) x [ra, rb) of the stress tile; the rest (closure
  // rows and columns, positions outside the grid) is the stress frame.
  int qa = max(0, 6 - X0), qb = min(sxn, n0 - 2 - X0), ra = max(0, 6 - Y0), rb = min(syn, n1 - 2 - Y0);
  if (qb <= qa || rb <= ra) qa = qb = 0, ra = rb = syn;
  qb = qa + ((qb - qa) & ~1);  // even width: the rectangle is done in pairs of positions
  if (qb == qa) ra = rb = syn;
  const int wq = qb - qa, nsframe = sxn * syn - wq * (rb - ra);
  // Of the central positions, those whose stencil reads only the own u (tile
  // columns and rows [4, w + 4)): [ia, ib) x [ja, jb), even width, computed
  // while the other CTAs finish the previous level.  In pair columns of the
  // central rectangle: [pa, pb) x [ja, jb); the rest of the rectangle (the
  // outer pairs) follows the halo ring.
  int ia = max(qa, 4), ib = min(qb, wx), ja = max(ra, 4), jb = min(rb, wy);
  ib = ib > ia ? ia + ((ib - ia) & ~1) : ia;
  const int wp = wq >> 1;
  int pa = (ia - qa) >> 1, pb = (ib - qa) >> 1, pja = ja - ra, pjb = jb - ra;
  if (pb <= pa || pjb <= pja) pa = pb = 0, pja = pjb = rb - ra;
  const int wpi = pb - pa, nouter = wp * (rb - ra) - wpi * (pjb - pja);
  // Own nodes on central rows and columns: the rectangle [xa, xb) x [ya, yb)
  // of the block (all unknowns, no closure, no boundary term); the others
  // (within 4 nodes of a side of the grid) are the special nodes.
  int xa = max(0, 4 - X0), xb = min(wx, n0 - 4 - X0), ya = max(0, 4 - Y0), yb = min(wy, n1 - 4 - Y0);
  if (xb <= xa || yb <= ya) xa = xb = 0, ya = yb = wy;
  xb = xa + ((xb - xa) & ~1);  // even width: regular nodes are updated in pairs
  if (xb == xa) ya = yb = wy;
  const int wr = xb - xa, nreg = wr * (yb - ya), nspec = wx * wy - nreg;
  const int wr2 = wr >> 1, npair = nreg >> 1;
  if (t < 24) tab[t] = c_sbp_f[t / 6][t % 6];

  {  // u^0 on the whole tile
    int lx = t % ux, ly = t / ux;
    const int rx = NT % ux, ry = NT / ux;
    for (; ly < uy; walk_next(lx, ly, ux, rx, ry)) {
      const int o = ubase + ly * npx + lx;
      su[ly * RS_UX + lx] = __ldcg(io.u0 + o);
      sv[ly * RS_UX + lx] = __ldcg(io.u0 + F + o);
    }
  }
  // walk of this thread's regular node pairs: l = t + NT k -> (xa + 2 (l % wr2), ya + l / wr2);
  // (ip, iy) below are relative to (xa / 2, ya)
  const int wrs = max(wr2, 1);
  const int ix0 = t % wrs, iy0 = t / wrs;
  const int qstep = NT / wrs, rstep = NT % wrs;
  float ac0[NP], ac1[NP], ac2[NP], ac3[NP];  // u, v of the pair's first node; u, v of its second
#pragma unroll
  for (int k = 0; k < NP; ++k) ac0[k] = ac1[k] = ac2[k] = ac3[k] = 0.f;
  RsLevel L;
  L.kt = (float)io.kt;
  L.w0 = (float)io.w0;
  bool alive = true;
  __syncthreads();

  for (int n = 0;; ++n) {
    if (wpi > 0) {  // central stresses that need only the own u, in pairs
      int pp = t % wpi, qy = ja + t / wpi;
      const int rx = NT % wpi, ry = NT / wpi;
      for (; qy < jb; walk_next(pp, qy, wpi, rx, ry))
        rs_stress_pair(io.lam, io.mu, npx, obase, qa + 2 * (pa + pp), qy);
    }
    if (n > 0) {
      if (!rs_wait(io.bar, (unsigned)n * gridDim.x, &s_ok, wait_ns)) {
        alive = false;
        break;
      }
      // halo ring of u^n from the neighbours' rims
      const float* xbuf = (n & 1) ? io.xbuf1 : io.xbuf0;
      {  // top and bottom strips: tile rows 0..3 and wy+4..wy+7, all columns
        int lx = t % ux, r = t / ux;
        const int rx = NT % ux, ry = NT / ux;
        for (; r < 2 * RS_HU; walk_next(lx, r, ux, rx, ry)) {
          const int ly = r < RS_HU ? r : wy + r;
          const int o = ubase + ly * npx + lx;
          su[ly * RS_UX + lx] = __ldcg(xbuf + o);
          sv[ly * RS_UX + lx] = __ldcg(xbuf + F + o);
        }
      }
      for (int i = t; i < 2 * RS_HU * wy; i += NT) {  // side strips: columns 0..3 and wx+4..wx+7
        const int c = i & (2 * RS_HU - 1), ly = RS_HU + (i >> 3);
        const int lx = c < RS_HU ? c : wx + c;
        const int o = ubase + ly * npx + lx;
        su[ly * RS_UX + lx] = __ldcg(xbuf + o);
        sv[ly * RS_UX + lx] = __ldcg(xbuf + F + o);
      }
    }
    __syncthreads();
    for (int j = t; j < nouter; j += NT) {  // the outer central pairs
      int pc, r;
      rs_frame_pos(j, wp, rb - ra, pa, pb, pja, pjb, pc, r);
      rs_stress_pair(io.lam, io.mu, npx, obase, qa + 2 * pc, ra + r);
    }
    for (int j = t; j < nsframe; j += NT) {  // the stress frame: general form
      int qx, qy;
      rs_frame_pos(j, sxn, syn, qa, qb, ra, rb, qx, qy);
      rs_stress_gen(io.lam, io.mu, n0, n1, npx, X0, Y0, obase, qx, qy, tab);
    }
    __syncthreads();
    // divergence and leapfrog/filter update of the own nodes
    L.first = n == 0;
    L.last = n == io.nsteps - 1;
    L.cosn = (float)io.cosn[n];
    L.wnew = (float)io.wnew[n];
    float* xo = (n & 1) ? io.xbuf0 : io.xbuf1;  // rims of u^{n+1}
    int ix = ix0, iy = iy0;
#pragma unroll
    for (int k = 0; k < NP; ++k) {  // regular node pairs: central differences only
      if (t + k * NT < npair) {
        const int jx = xa + 2 * ix, jy = ya + iy;
        const int ps = (jy + RS_HS) * RS_SX + (jx + RS_HS);  // even
        const float2* SXX = reinterpret_cast<const float2*>(sxx + ps);
        const float2* SYY = reinterpret_cast<const float2*>(syy + ps);
        const float2* SXY = reinterpret_cast<const float2*>(sxy + ps);
        constexpr int RS2 = RS_SX / 2;
        const float2 xa_ = SXX[-1], xb_ = SXX[0], xc_ = SXX[1];
        const float2 ya_ = SXY[-1], yb_ = SXY[0], yc_ = SXY[1];
        const float kxu0 = c4(xa_.x, xa_.y, xb_.y, xc_.x), kxu1 = c4(xa_.y, xb_.x, xc_.x, xc_.y);
        const float kxv0 = c4(ya_.x, ya_.y, yb_.y, yc_.x), kxv1 = c4(ya_.y, yb_.x, yc_.x, yc_.y);
        const float2 sm2 = SXY[-2 * RS2], sm1 = SXY[-RS2], sp1 = SXY[RS2], sp2 = SXY[2 * RS2];
        const float2 tm2 = SYY[-2 * RS2], tm1 = SYY[-RS2], tp1 = SYY[RS2], tp2 = SYY[2 * RS2];
        const float kyu0 = c4(sm2.x, sm1.x, sp1.x, sp2.x), kyu1 = c4(sm2.y, sm1.y, sp1.y, sp2.y);
        const float kyv0 = c4(tm2.x, tm1.x, tp1.x, tp2.x), kyv1 = c4(tm2.y, tm1.y, tp1.y, tp2.y);
        const float ku0 = -kxu0 - kyu0, ku1 = -kxu1 - kyu1;
        const float kv0 = -kxv0 - kyv0, kv1 = -kxv1 - kyv1;
        const int o = obase + jy * npx + jx;
        const float r0 = __ldg(io.irh2 + o), r1 = __ldg(io.irh2 + o + 1);
        float au0 = ku0 * r0, av0 = kv0 * r0, au1 = ku1 * r1, av1 = kv1 * r1;
        if (io.frho) {
          au0 += __ldg(io.frho + o) * L.cosn;
          au1 += __ldg(io.frho + o + 1) * L.cosn;
          av0 += __ldg(io.frho + F + o) * L.cosn;
          av1 += __ldg(io.frho + F + o + 1) * L.cosn;
        }
        const int pu = (jy + RS_HU) * RS_UX + (jx + RS_HU);  // even
        const int pd = jy * RS_BXMAX + jx;                   // even
        float2* Up = reinterpret_cast<float2*>(su + pu);
        float2* Vp = reinterpret_cast<float2*>(sv + pu);
        float2* Dup = reinterpret_cast<float2*>(rs_smem + RS_OFF_DU + pd);
        float2* Dvp = reinterpret_cast<float2*>(rs_smem + RS_OFF_DV + pd);
        const float2 uu = *Up, uv = *Vp;
        float2 du, dv;
        if (L.first) {
          du = make_float2(-0.5f * L.kt * au0, -0.5f * L.kt * au1);
          dv = make_float2(-0.5f * L.kt * av0, -0.5f * L.kt * av1);
        } else {
          const float2 d0 = *Dup, d1 = *Dvp;
          du = make_float2(d0.x - L.kt * au0, d0.y - L.kt * au1);
          dv = make_float2(d1.x - L.kt * av0, d1.y - L.kt * av1);
        }
        const float2 nu_ = make_float2(uu.x + du.x, uu.y + du.y), nv_ = make_float2(uv.x + dv.x, uv.y + dv.y);
        if (L.first) {
          ac0[k] = L.w0 * uu.x + L.wnew * nu_.x;
          ac1[k] = L.w0 * uv.x + L.wnew * nv_.x;
          ac2[k] = L.w0 * uu.y + L.wnew * nu_.y;
          ac3[k] = L.w0 * uv.y + L.wnew * nv_.y;
        } else {
          ac0[k] += L.wnew * nu_.x;
          ac1[k] += L.wnew * nv_.x;
          ac2[k] += L.wnew * nu_.y;
          ac3[k] += L.wnew * nv_.y;
        }
        *Dup = du;
        *Dvp = dv;
        if (!L.last) {
          *Up = nu_;
          *Vp = nv_;
          const bool rowrim = jy < RS_HU || jy >= wy - RS_HU;
          if (rowrim || jx < RS_HU || jx >= wx - RS_HU) {
            xo[o] = nu_.x;
            xo[F + o] = nv_.x;
          }
          if (rowrim || jx + 1 < RS_HU || jx + 1 >= wx - RS_HU) {
            xo[o + 1] = nu_.y;
            xo[F + o + 1] = nv_.y;
          }
        }
      }
      walk_next(ix, iy, wr2, rstep, qstep);
    }
    for (int j = t; j < nspec; j += NT) {  // special nodes: general form, accumulators in shared memory
      int jx, jy;
      rs_frame_pos(j, wx, wy, xa, xb, ya, yb, jx, jy);
      const int x = X0 + jx, y = Y0 + jy;
      const bool unk = (x > 0 || g.lo_free[0]) && (x < n0 - 1 || g.hi_free[0]) && (y > 0 || g.lo_free[1]) &&
                       (y < n1 - 1 || g.hi_free[1]);
      if (unk) {
        float au, av;
        rs_accel_gen(g, io.irh2, io.frho, F, X0, Y0, obase, jx, jy, L, tab, au, av);
        rs_update(jx, jy, au, av, L, sacc[2 * j], sacc[2 * j + 1]);
      }
      if (!L.last && (jx < RS_HU || jx >= wx - RS_HU || jy < RS_HU || jy >= wy - RS_HU)) {
        const int o = obase + jy * npx + jx;
        const int pu = (jy + RS_HU) * RS_UX + (jx + RS_HU);
        xo[o] = su[pu];
        xo[F + o] = sv[pu];
      }
    }
    if (L.last) break;
    __syncthreads();  // this level's u and rims are written
    rs_arrive(io.bar);
  }
  // accumulators of the own unknowns (NaN when the barrier gave up)
  const float nanv = __int_as_float(0x7fc00000);
  int ix = ix0, iy = iy0;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    if (t + k * NT < npair) {
      const int o = obase + (ya + iy) * npx + (xa + 2 * ix);
      io.acc[o] = alive ? ac0[k] : nanv;
      io.acc[F + o] = alive ? ac1[k] : nanv;
      io.acc[o + 1] = alive ? ac2[k] : nanv;
      io.acc[F + o + 1] = alive ? ac3[k] : nanv;
    }
    walk_next(ix, iy, wr2, rstep, qstep);
  }
  __syncthreads();  // the special accumulators were written by other threads
  for (int j = t; j < nspec; j += NT) {
    int jx, jy;
    rs_frame_pos(j, wx, wy, xa, xb, ya, yb, jx, jy);
    const int x = X0 + jx, y = Y0 + jy;
    if ((x > 0 || g.lo_free[0]) && (x < n0 - 1 || g.hi_free[0]) && (y > 0 || g.lo_free[1]) &&
        (y < n1 - 1 || g.hi_free[1])) {
      const int o = obase + jy * npx + jx;
      io.acc[o] = alive ? sacc[2 * j] : nanv;
      io.acc[F + o] = alive ? sacc[2 * j + 1] : nanv;
    }
  }
}

static size_t resident_smem() { return sizeof(float) * (size_t)RS_FLOATS; }

// Opt the kernel in to the device's largest dynamic shared memory (the same
// value for every context, so plans of different sizes never undo each
// other; set before any launch or capture) and report CTAs per SM at smem.
template <int NT, int NP>
static cudaError_t resident_prepare(int smem_max, size_t smem, int* per_sm) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, step2d_o4_resident<NT, NP>);
  if (e != cudaSuccess) return e;
  const int dyn_max = smem_max - (int)fa.sharedSizeBytes;  // static + dynamic <= opt-in limit
  if ((long long)smem > dyn_max) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(step2d_o4_resident<NT, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, step2d_o4_resident<NT, NP>, NT, smem);
}

static cudaError_t resident_prepare_shape(int shape, int smem_max, size_t smem, int* per_sm) {
  switch (shape) {
    case 0: return resident_prepare<RS_SHAPE_THREADS[0], RS_SHAPE_PAIRS[0]>(smem_max, smem, per_sm);
    case 1: return resident_prepare<RS_SHAPE_THREADS[1], RS_SHAPE_PAIRS[1]>(smem_max, smem, per_sm);
    case 2: return resident_prepare<RS_SHAPE_THREADS[2], RS_SHAPE_PAIRS[2]>(smem_max, smem, per_sm);
    default: return cudaErrorInvalidValue;
  }
}

ResidentPlan plan_resident_o4(const Geom& g, int shape) {
  ResidentPlan best;
  if (g.dim != 2 || g.nrhs < 1 || g.field >= (1LL << 31) || shape < 0 || shape >= RS_SHAPES) return best;
  int dev = 0, sms = 0, smem_max = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) {
    cudaGetLastError();
    return best;
  }
  // every CTA of a launch must be resident at once
  int per_sm = 0;
  const cudaError_t e = resident_prepare_shape(shape, smem_max, resident_smem(), &per_sm);
  const bool verbose = getenv("EWH_VERBOSE") != nullptr;
  if (e != cudaSuccess || per_sm < 1) {
    if (verbose) fprintf(stderr, "ewh: resident shape %d unusable (%s)\n", shape, cudaGetErrorString(e));
    cudaGetLastError();
    return best;
  }
  const int ctas = per_sm * sms;  // co-resident CTAs of one launch
  const int R = g.nrhs;
  const long long cap = 2LL * RS_SHAPE_THREADS[shape] * RS_SHAPE_PAIRS[shape];
  const int n0 = g.n[0], n1 = g.n[1];
  // Blocks that hold x-closure columns (the first and last along x) take
  // about RS_EDGE_COST longer per node (a few lanes of their warps diverge):
  // they get proportionally fewer columns, so all CTAs reach each barrier
  // together.
  constexpr double RS_EDGE_COST = 1.1;
  // A level costs a CTA about its tile work plus a fixed part (the barrier,
  // the halo exchange) worth RS_LEVEL_FIXED tile positions.  With several
  // right-hand sides, each launch carries a group of rg of them (rg x px x py
  // CTAs, all co-resident) and the groups run one after another: the cost is
  // the number of groups times the slowest CTA's level.
  constexpr double RS_LEVEL_FIXED = 3000.0;
  double best_cost = -1.0;
  for (int px = 1; px <= ctas && px <= n0 / 8; ++px) {
    int bx, ex, last;
    if (px == 1) {
      bx = ex = last = n0;
    } else {
      bx = px == 2 ? (n0 + 1) / 2 : (int)std::ceil(n0 / (px - 2 + 2.0 / RS_EDGE_COST));
      ex = px == 2 ? bx : (n0 - (px - 2) * bx) / 2;
      last = n0 - ex - (px - 2) * bx;
    }
    if (ex < 8 || last < 8 || bx > RS_BXMAX || ex > RS_BXMAX || last > RS_BXMAX) continue;
    const int wmax = std::max(bx, std::max(ex, last));
    for (int py = 1; px * py <= ctas && py <= n1 / 8; ++py) {
      const int by = (n1 + py - 1) / py;
      const int pya = (n1 + by - 1) / by;
      if (n1 - (pya - 1) * by < 8) continue;
      if ((long long)wmax * by > cap || by > RS_BYMAX) continue;
      // nodes within 4 of a side of the grid, per block, fit their shared accumulators
      auto spec = [&](int X0, int w, int Y0, int h) {
        const int a = std::max(0, 4 - X0), b0 = std::min(w, n0 - 4 - X0), b = b0 > a ? a + ((b0 - a) & ~1) : b0;
        const int c = std::max(0, 4 - Y0), d = std::min(h, n1 - 4 - Y0);
        return w * h - ((b > a && d > c) ? (b - a) * (d - c) : 0);
      };
      bool fits = true;
      for (int cy = 0; cy < pya && fits; ++cy)
        for (int cx = 0; cx < px && fits; ++cx) {
          const int X0 = cx == 0 ? 0 : ex + (cx - 1) * bx;
          const int w = cx == 0 ? ex : std::min(bx, n0 - X0);
          fits = spec(X0, w, cy * by, std::min(by, n1 - cy * by)) <= RS_SPECIAL_MAX;
        }
      if (!fits) continue;
      const size_t sm = resident_smem();
      if (sm > (size_t)smem_max) continue;
      // per-CTA work (u tile + stress tile) of the slowest block
      auto work = [&](int w) { return (double)(w + 2 * RS_HU) * (by + 2 * RS_HU) + (double)(w + 2 * RS_HS) * (by + 2 * RS_HS); };
      const double level = px == 1 ? work(bx) * RS_EDGE_COST
                                   : std::max(work(bx), RS_EDGE_COST * work(std::max(ex, last)));
      const int nb = px * pya;
      const int rg0 = std::min(R, ctas / nb);
      if (rg0 < 1) continue;
      const int groups = (R + rg0 - 1) / rg0;
      const double cost = groups * (level + RS_LEVEL_FIXED);
      if (best_cost < 0 || cost < best_cost) {
        best_cost = cost;
        best.ok = 1;
        best.shape = shape;
        best.px = px;
        best.py = pya;
        best.bx = bx;
        best.ex = ex;
        best.by = by;
        best.smem = sm;
        best.groups = groups;
        best.rg = (R + groups - 1) / groups;  // balanced groups
      }
    }
  }
  if (!best.ok) return best;
  if (verbose)
    fprintf(stderr,
            "ewh: resident shape %d: %d x %d CTAs of %d (first %d) x %d nodes per rhs, %d rhs per launch in %d "
            "launches, %zu B shared\n",
            shape, best.px, best.py, best.bx, best.ex, best.by, best.rg, best.groups, best.smem);
  return best;
}

template <int NT, int NP>
static cudaError_t resident_launch(const Geom& g, const ResidentPlan& p, const ResidentIO& io, int nr,
                                   cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nr * p.px * p.py);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = p.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ResidentShape sh{p.px, p.bx, p.by, p.ex, p.px * p.py};
  return cudaLaunchKernelEx(&cfg, step2d_o4_resident<NT, NP>, g, sh, io);
}

// The groups of right-hand sides one after another, each one cooperative
// launch (its barrier words zeroed first).
cudaError_t launch_resident_o4(const Geom& g, const ResidentPlan& p, const ResidentIO& io, cudaStream_t st) {
  if (!p.ok || g.dim != 2 || io.nsteps < 1 || p.rg < 1 || (long long)p.rg * p.groups < g.nrhs)
    return cudaErrorInvalidValue;
  for (int k = 0; k < p.groups; ++k) {
    const int r0 = k * p.rg, nr = std::min(p.rg, g.nrhs - r0);
    if (nr < 1) break;
    ResidentIO gi = io;
    const long long ro = (long long)r0 * 2 * g.field;
    gi.u0 += ro;
    gi.xbuf0 += ro;
    gi.xbuf1 += ro;
    gi.acc += ro;
    if (gi.frho) gi.frho += ro;
    cudaError_t e = cudaMemsetAsync(io.bar, 0, 2 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    switch (p.shape) {
      case 0: e = resident_launch<RS_SHAPE_THREADS[0], RS_SHAPE_PAIRS[0]>(g, p, gi, nr, st); break;
      case 1: e = resident_launch<RS_SHAPE_THREADS[1], RS_SHAPE_PAIRS[1]>(g, p, gi, nr, st); break;
      case 2: e = resident_launch<RS_SHAPE_THREADS[2], RS_SHAPE_PAIRS[2]>(g, p, gi, nr, st); break;
      default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template cudaError_t launch_step<float>(const Geom&, int, const WaveFields<float>&, StepMode,
                                        const StepScalars&, cudaStream_t, long long*);
template cudaError_t launch_step<double>(const Geom&, int, const WaveFields<double>&, StepMode,
                                         const StepScalars&, cudaStream_t, long long*);
template cudaError_t launch_minvK<float>(const Geom&, int, const float*, float*, const float*, const float*,
                                         const float*, float*, cudaStream_t, long long*, const float*);
template cudaError_t launch_minvK<double>(const Geom&, int, const double*, double*, const double*,
                                          const double*, const double*, double*, cudaStream_t, long long*,
                                          const double*);

}  // namespace ewh
