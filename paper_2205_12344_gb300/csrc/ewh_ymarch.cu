// Order 4 (SBP), 2D, FP32: one fused launch per leapfrog level that marches
// along y.  The level is the time-corrected explicit scheme of Section 4.3
// (eq. elastic-time-explicit-corrected) in increment form with the trapezoid
// accumulation of eq. (qoper), for the order-4 operator
//   M^{-1} K u = (1 / (rho h^2)) sum_a [ -D_a sigma_{.a} + H_a^{-1} B_a sigma_{.a} ].
//
// One warp per CTA owns a strip of 60 unknown columns (30 node pairs) and a
// range of rows of one right-hand side, and walks the rows upwards.  Per row
//   - u^n (2 components) arrives on the strip +- 4 nodes through a bulk-tensor
//     (TMA) load issued two rows ahead into a ring of 8 row buffers (one
//     complete-tx mbarrier each);
//   - every lane forms the scaled stresses 12 sigma at one node pair of the
//     strip +- 2 nodes: (xx, xy) into a row buffer for the x differences,
//     (xy, yy) of the own pairs into a ring of 8 rows for the y differences;
//   - the own lanes form -D_x sigma_{.x} (+ the x boundary terms) into a ring
//     of 6 pending rows, and for every output row whose y stencil is complete
//     add -D_y sigma_{.y} (+ the y boundary terms) and apply the leapfrog /
//     filter update (8-byte loads and stores of node pairs).
// The stresses never leave the chip.  A CTA holds about 13 KB of shared
// memory, so 16 CTAs (warps) share an SM; a persistent grid splits the
// (right-hand side, strip, row) work into equal contiguous shares of at
// least EWH_YM_ROWS (32) rows, so many right-hand sides fill the GPU.  The rows near the y sides follow the exact reach of
// the SBP closure rows (the schedule of ewh_zmarch.cu, along y); the strips'
// x closures use the per-class tap tables (no lane divergence).  Waits on the
// mbarriers are bounded by the context's wait limit; a CTA that gives up
// counts itself in ctl[4], fills its remaining accumulators with NaN and
// returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "ewh_internal.cuh"
#include "ewh_march.cuh"

namespace ewh {

namespace {

constexpr int YM_TX = 60;   // own columns per strip (30 pairs)
constexpr int YM_UX = 68;   // u row: x from X0 - 4 (the bulk-tensor box width)
constexpr int YM_SX = 64;   // stress row: x from X0 - 2 (32 pairs = the warp)
constexpr int YM_RU = 8;    // u row ring
constexpr int YM_RS = 8;    // (xy, yy) stress ring of the own pairs
constexpr int YM_RP = 6;    // pending x-divergence ring
constexpr int YM_PREF = 2;  // u rows requested ahead of the march
constexpr int YM_USLOT = 160;             // floats per u slot (2 x 68, padded to 640 bytes)
constexpr int YM_OFF_SZ = YM_RU * YM_USLOT;
constexpr int YM_OFF_PD = YM_OFF_SZ + YM_RS * 2 * YM_TX;
constexpr int YM_OFF_SIP = YM_OFF_PD + YM_RP * 2 * YM_TX;
constexpr int YM_OFF_TAB = YM_OFF_SIP + 2 * YM_SX;
constexpr int YM_OFF_CLS = YM_OFF_TAB + 24;
constexpr int YM_FLOATS = YM_OFF_CLS + 8 * ZM_CLASSES;
constexpr size_t YM_BYTES = 128 + sizeof(float) * YM_FLOATS + sizeof(uint64_t) * YM_RU;
constexpr unsigned YM_TX_BYTES = sizeof(float) * 2 * YM_UX;  // one bulk-tensor box (2 components)
static_assert(YM_USLOT % 32 == 0 && YM_USLOT >= 2 * YM_UX, "u slots stay 128-byte aligned");
static_assert(YM_OFF_CLS % 4 == 0 && YM_FLOATS % 2 == 0, "table and mbarrier alignment");

struct YmScalars {
  float tab12[24];  // 12 x SBP_CLOSURE
  float kt144;      // c dt^2 / 144
  float w0, wnew;   // trapezoid weights of level 0 (first level only) and of the new level
  float fcos144;    // 144 cos(w t_n)
  float bt12;       // 12 * 48 / 17: H^{-1} B in the scaled arithmetic
  int shx;         // strip origins: off[0] - shx + 60 k (see zm_shift)
  // 12 D at a node of class k as four taps (offsets, weights; see zm_class_taps)
  int toff[4 * ZM_CLASSES];
  float tcf[4 * ZM_CLASSES];
};

struct YmOperands {  // update operands of one own pair at one output row
  float2 d[2], a[2], f[2], irh;
};

// 2D component offset of node (x, y)
__device__ __forceinline__ int ym_off(const Geom& g, int x, int y) { return (y + PAD) * g.np[0] + x + g.padx; }

template <bool FORCED>
__device__ __forceinline__ void ym_load_ops(const float* D, const float* A, const float* R, const float* irh2, int o,
                                            int F, bool v0, bool v1, YmOperands& op) {
  if (v0 && v1) {  // 8-byte aligned: the padded x of a pair's first node is even
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      op.d[c] = __ldcs(reinterpret_cast<const float2*>(D + o + c * F));
      op.a[c] = __ldcs(reinterpret_cast<const float2*>(A + o + c * F));
      if (FORCED) op.f[c] = __ldg(reinterpret_cast<const float2*>(R + o + c * F));
    }
    op.irh = __ldg(reinterpret_cast<const float2*>(irh2 + o));
  } else {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      op.d[c] = make_float2(v0 ? D[o + c * F] : 0.f, v1 ? D[o + c * F + 1] : 0.f);
      op.a[c] = make_float2(v0 ? A[o + c * F] : 0.f, v1 ? A[o + c * F + 1] : 0.f);
      if (FORCED) op.f[c] = make_float2(v0 ? R[o + c * F] : 0.f, v1 ? R[o + c * F + 1] : 0.f);
    }
    op.irh = make_float2(v0 ? irh2[o] : 0.f, v1 ? irh2[o + 1] : 0.f);
  }
}

__device__ __forceinline__ void ym_load_lm(const float* lam, const float* mu, int o, bool g0, bool g1, float2& l,
                                           float2& m) {
  if (g0 && g1) {
    l = __ldg(reinterpret_cast<const float2*>(lam + o));
    m = __ldg(reinterpret_cast<const float2*>(mu + o));
    return;
  }
  l = m = make_float2(0.f, 0.f);
  if (g0) l.x = __ldg(lam + o), m.x = __ldg(mu + o);
  if (g1) l.y = __ldg(lam + o + 1), m.y = __ldg(mu + o + 1);
}

// Request one u row (2 components of box YM_UX x 1 at padded (cx, cy), components
// cc, cc + 1) into dst; completion is counted on bar.
__device__ __forceinline__ void ym_issue(const CUtensorMap* tm, float* dst, uint64_t* bar, int cx, int cy, int cc) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(YM_TX_BYTES)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(cx), "r"(cy), "r"(cc), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool ym_unknown_x(const Geom& g, int x) { return x >= g.off[0] && x < g.off[0] + g.nu[0]; }

constexpr unsigned YM_ALL = 0xffffffffu;

template <int MODE, bool FORCED>
__global__ void __launch_bounds__(32) step2d_o4_ym(Geom g, WaveFields<float> f, YmScalars sc, unsigned* ctl,
                                                   const __grid_constant__ CUtensorMap tmu) {
  extern __shared__ unsigned char ym_raw[];
  // 128-byte aligned base, offset from the shared array itself (shared address space)
  float* const sm = reinterpret_cast<float*>(ym_raw + ((128u - (smem_u32(ym_raw) & 127u)) & 127u));
  uint64_t* const bar = reinterpret_cast<uint64_t*>(sm + YM_FLOATS);
  float* const tab = sm + YM_OFF_TAB;
  float* const sip = sm + YM_OFF_SIP;
  int* const toff = reinterpret_cast<int*>(sm + YM_OFF_CLS);
  float* const tcf = sm + YM_OFF_CLS + 4 * ZM_CLASSES;
  const int t = threadIdx.x;
  if (t == 0) {  // static indices: the parameter arrays stay in the constant bank
#pragma unroll
    for (int k = 0; k < 24; ++k) tab[k] = sc.tab12[k];
#pragma unroll
    for (int k = 0; k < 4 * ZM_CLASSES; ++k) toff[k] = sc.toff[k], tcf[k] = sc.tcf[k];
    for (int k = 0; k < YM_RU; ++k) mbar_init(bar + k, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  zm_pdl_wait();
  zm_pdl_trigger();
  const unsigned long long wait_ns = *reinterpret_cast<const volatile unsigned long long*>(ctl + 2);

  const int n0 = g.n[0], n1 = g.n[1], ny = g.nu[1];
  const int ntx = (g.nu[0] + sc.shx + YM_TX - 1) / YM_TX;
  const long long W = (long long)ntx * ny * g.nrhs;
  const long long wbeg = W * blockIdx.x / gridDim.x, wend = W * (blockIdx.x + 1) / gridDim.x;
  // lane t: stress pair (X0 - 2 + 2t, + 1); lanes 1..30 also own the pair i = t - 1
  const bool own = t >= 1 && t <= 30;
  const int i = t - 1;
  const int F = (int)g.field, NPX = g.np[0];
  const float BT = sc.bt12;
  unsigned phase = 0;  // parity of the next completion of each u slot's mbarrier
  bool alive = true;
  long long w = wbeg;

  while (w < wend && alive) {
    // ---- segment: strip (rhs, tx), output rows [ya, yb)
    const long long tile = w / ny;
    const int yi = (int)(w - tile * ny);
    const int ycount = (int)((wend - w) < (long long)(ny - yi) ? (wend - w) : (long long)(ny - yi));
    w += ycount;
    const int rhs = (int)(tile / ntx);
    const int X0 = g.off[0] - sc.shx + YM_TX * (int)(tile - (long long)rhs * ntx);
    const int ya = g.off[1] + yi, yb = ya + ycount;
    // stress rows [slo, shi] the outputs read; u rows [ulo, uhi] those read
    const int slo = min(zm_lo(ya, n1), zm_lo(yb - 1, n1)), shi = max(zm_hi(ya, n1), zm_hi(yb - 1, n1));
    const int ulo = min(zm_lo(slo, n1), zm_lo(shi, n1)), uhi = max(zm_hi(slo, n1), zm_hi(shi, n1));
    const int hs0 = zm_hi(slo, n1), ho0 = zm_hi(ya, n1);
    const int cx = X0 - 4 + g.padx, cc = 2 * rhs;  // bulk-tensor x: a multiple of 4 (Geom::padx, shx)
    __syncwarp();  // every read of the rings by the previous segment is done
    if (t == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      for (int k = ulo; k <= uhi && k < ulo + YM_PREF; ++k)
        ym_issue(&tmu, sm + (k & (YM_RU - 1)) * YM_USLOT, bar + (k & (YM_RU - 1)), cx, k + PAD, cc);
    }
    const int sx = X0 - 2 + 2 * t;
    const bool sg0 = sx >= 0 && sx < n0, sg1 = sx + 1 >= 0 && sx + 1 < n0;
    const int cx0 = zm_class(sx, n0), cx1 = zm_class(sx + 1, n0);
    const bool wx = __any_sync(YM_ALL, cx0 != 4 || cx1 != 4);  // a lane on an x closure row
    const bool ov0 = own && ym_unknown_x(g, sx), ov1 = own && ym_unknown_x(g, sx + 1);
    const int so = ym_off(g, sx, 0);  // row y adds y * NPX
    const long long ro = (long long)rhs * 2 * g.field;
    const float* const Dr = f.delta + ro;
    const float* const Ar = f.acc + ro;
    const float* const Rr = FORCED ? f.frho + ro : nullptr;
    float* const Dw = f.delta + ro;
    float* const Aw = f.acc + ro;
    float* const Uw = f.u_next + ro;
    float2 lm_l, lm_m;
    int lm_row = slo;
    ym_load_lm(f.lam, f.mu, so + slo * NPX, sg0, sg1, lm_l, lm_m);
    YmOperands op;
    int op_row = -1;
    if (ov0 || ov1) {
      ym_load_ops<FORCED>(Dr, Ar, Rr, f.irh2, so + ya * NPX, F, ov0, ov1, op);
      op_row = ya;
    }

    int next_s = slo, next_o = ya, jfail = uhi + 1;
    bool wait_bad = false;
    for (int j = ulo; j <= uhi; ++j) {
      // ---- wait for u row j (bounded)
      {
        const int k = j & (YM_RU - 1);
        const unsigned par = (phase >> k) & 1u;
        bool ok = wait_ns != 0ull;
        if (ok && !mbar_try(bar + k, par)) {
          const unsigned long long t0 = zm_ns();
          while (!mbar_try(bar + k, par)) {
            if (zm_ns() - t0 > wait_ns) {
              ok = false;
              break;
            }
          }
        }
        if (ok) phase ^= 1u << k;
        wait_bad = !ok;  // the lanes agree at the next vote
      }
      bool any_sigma = false, failed = false;
      // the last stress row complete at this step (prefix maximum of the reach)
      const int s_last = zm_last_ready(next_s, shi, hs0, j, n1);
      for (; next_s <= s_last;) {
        const int ys = next_s;
        if (lm_row != ys) {
          ym_load_lm(f.lam, f.mu, so + ys * NPX, sg0, sg1, lm_l, lm_m);
          lm_row = ys;
        }
        const float* U0 = sm + (ys & (YM_RU - 1)) * YM_USLOT;
        const bool yin = ys >= 4 && ys <= n1 - 5;  // uniform per row
        const int lx = 2 + 2 * t;                  // u row position of node sx
        float d0[2][2], d1[2][2];                  // d[c][a] = 12 D_a u_c
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int o = c * YM_UX + lx;
          const float* Uc = U0 + o;
          const float2 a = ld2(Uc - 2), b = ld2(Uc), e = ld2(Uc + 2);
          d0[c][0] = c4u(a.x, a.y, b.y, e.x);
          d1[c][0] = c4u(a.y, b.x, e.x, e.y);
          if (yin) {
            const float2 m2 = ld2(sm + ((ys - 2) & (YM_RU - 1)) * YM_USLOT + o);
            const float2 m1 = ld2(sm + ((ys - 1) & (YM_RU - 1)) * YM_USLOT + o);
            const float2 p1 = ld2(sm + ((ys + 1) & (YM_RU - 1)) * YM_USLOT + o);
            const float2 p2 = ld2(sm + ((ys + 2) & (YM_RU - 1)) * YM_USLOT + o);
            d0[c][1] = c4u(m2.x, m1.x, p1.x, p2.x);
            d1[c][1] = c4u(m2.y, m1.y, p1.y, p2.y);
          } else {
            d0[c][1] = zm_closure12([&](int k) { return sm[((ys + k) & (YM_RU - 1)) * YM_USLOT + o]; }, ys, n1, tab);
            d1[c][1] =
                zm_closure12([&](int k) { return sm[((ys + k) & (YM_RU - 1)) * YM_USLOT + o + 1]; }, ys, n1, tab);
          }
        }
        if (wx) {  // x closure rows: every lane with its own class taps
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const float* Uc = U0 + c * YM_UX + lx;
            d0[c][0] = zm_d12t(Uc, 1, cx0, toff, tcf);
            d1[c][0] = zm_d12t(Uc + 1, 1, cx1, toff, tcf);
          }
        }
        // 12 sigma: xx, yy, xy
        const float dv0 = d0[0][0] + d0[1][1], dv1 = d1[0][0] + d1[1][1];
        float xx0 = lm_l.x * dv0 + 2.0f * lm_m.x * d0[0][0], xx1 = lm_l.y * dv1 + 2.0f * lm_m.y * d1[0][0];
        float yy0 = lm_l.x * dv0 + 2.0f * lm_m.x * d0[1][1], yy1 = lm_l.y * dv1 + 2.0f * lm_m.y * d1[1][1];
        float xy0 = lm_m.x * (d0[0][1] + d0[1][0]), xy1 = lm_m.y * (d1[0][1] + d1[1][0]);
        if (!sg0) xx0 = yy0 = xy0 = 0.f;
        if (!sg1) xx1 = yy1 = xy1 = 0.f;
        st2(sip + 2 * t, xx0, xx1);
        st2(sip + YM_SX + 2 * t, xy0, xy1);
        if (own) {  // (xy, yy) of the own pair into the ring
          float* SZ = sm + YM_OFF_SZ + (ys & (YM_RS - 1)) * 2 * YM_TX + 2 * i;
          st2(SZ, xy0, xy1);
          st2(SZ + YM_TX, yy0, yy1);
        }
        if (ys + 1 <= shi) {
          ym_load_lm(f.lam, f.mu, so + (ys + 1) * NPX, sg0, sg1, lm_l, lm_m);
          lm_row = ys + 1;
        }
        __syncwarp();  // the stress row is complete
        if (__any_sync(YM_ALL, wait_bad)) {
          failed = true;
          break;
        }
        any_sigma = true;
        if (ys >= ya && ys < yb && (ov0 || ov1)) {
          // x part of -D sigma + H^{-1} B sigma: D_x sigma_xx (x), D_x sigma_xy (y)
          float k0[2], k1[2];
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const float* Sx = sip + c * YM_SX + 2 * t;
            float q0, q1;
            if (wx) {
              q0 = zm_d12t(Sx, 1, cx0, toff, tcf);
              q1 = zm_d12t(Sx + 1, 1, cx1, toff, tcf);
            } else {
              const float2 a = ld2(Sx - 2), b = ld2(Sx), e = ld2(Sx + 2);
              q0 = c4u(a.x, a.y, b.y, e.x);
              q1 = c4u(a.y, b.x, e.x, e.y);
            }
            k0[c] = -q0;
            k1[c] = -q1;
            if (wx) {  // boundary terms on free x sides (nodes on the side itself)
              if (sx == 0) k0[c] -= BT * Sx[0];
              if (sx == n0 - 1) k0[c] += BT * Sx[0];
              if (sx + 1 == n0 - 1) k1[c] += BT * Sx[1];
            }
          }
          float* PD = sm + YM_OFF_PD + (ys % YM_RP) * 2 * YM_TX + 2 * i;
          st2(PD, k0[0], k1[0]);
          st2(PD + YM_TX, k0[1], k1[1]);
        }
        ++next_s;
        if (next_s <= s_last) __syncwarp();  // another row follows: its stresses overwrite sip
      }
      if (!any_sigma && !failed) {
        __syncwarp();
        failed = __any_sync(YM_ALL, wait_bad) != 0;
      }
      if (failed) {  // a wait gave up: every lane stops here
        alive = false;
        jfail = j;
        break;
      }
      // ---- output rows whose stress rows all exist
      const int o_last = zm_last_ready(next_o, yb - 1, ho0, next_s - 1, n1);
      for (; next_o <= o_last; ++next_o) {
        const int yo = next_o;
        if (!(ov0 || ov1)) continue;
        if (op_row != yo) ym_load_ops<FORCED>(Dr, Ar, Rr, f.irh2, so + yo * NPX, F, ov0, ov1, op);
        const float* PD = sm + YM_OFF_PD + (yo % YM_RP) * 2 * YM_TX + 2 * i;
        float k0[2], k1[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const float2 pd = ld2(PD + c * YM_TX);
          k0[c] = pd.x;
          k1[c] = pd.y;
        }
        // y part: D_y sigma_xy (x), D_y sigma_yy (y)
        if (yo >= 4 && yo <= n1 - 5) {
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int o = YM_OFF_SZ + c * YM_TX + 2 * i;
            const float2 m2 = ld2(sm + ((yo - 2) & (YM_RS - 1)) * 2 * YM_TX + o);
            const float2 m1 = ld2(sm + ((yo - 1) & (YM_RS - 1)) * 2 * YM_TX + o);
            const float2 p1 = ld2(sm + ((yo + 1) & (YM_RS - 1)) * 2 * YM_TX + o);
            const float2 p2 = ld2(sm + ((yo + 2) & (YM_RS - 1)) * 2 * YM_TX + o);
            k0[c] -= c4u(m2.x, m1.x, p1.x, p2.x);
            k1[c] -= c4u(m2.y, m1.y, p1.y, p2.y);
          }
        } else {
#pragma unroll
          for (int c = 0; c < 2; ++c) {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const int o = YM_OFF_SZ + c * YM_TX + 2 * i + e;
              auto v = [&](int k) { return sm[((yo + k) & (YM_RS - 1)) * 2 * YM_TX + o]; };
              float kc = -zm_closure12(v, yo, n1, tab);
              if (yo == 0) kc -= BT * v(0);  // boundary terms on free y sides
              else if (yo == n1 - 1) kc += BT * v(0);
              if (e) k1[c] += kc;
              else k0[c] += kc;
            }
          }
        }
        // leapfrog / filter update of the pair (increment form)
        const float* Uo = sm + (yo & (YM_RU - 1)) * YM_USLOT + 4 + 2 * i;
        const int p = so + yo * NPX;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const float2 u = ld2(Uo + c * YM_UX);
          float a0 = k0[c] * op.irh.x, a1 = k1[c] * op.irh.y;
          if (FORCED) {
            a0 += op.f[c].x * sc.fcos144;
            a1 += op.f[c].y * sc.fcos144;
          }
          float dd0, dd1;
          if (MODE == STEP_FIRST) {
            dd0 = -0.5f * sc.kt144 * a0;
            dd1 = -0.5f * sc.kt144 * a1;
          } else {
            dd0 = op.d[c].x - sc.kt144 * a0;
            dd1 = op.d[c].y - sc.kt144 * a1;
          }
          const float un0 = u.x + dd0, un1 = u.y + dd1;
          float ac0, ac1;
          if (MODE == STEP_FIRST) {
            ac0 = sc.w0 * u.x + sc.wnew * un0;
            ac1 = sc.w0 * u.y + sc.wnew * un1;
          } else {
            ac0 = op.a[c].x + sc.wnew * un0;
            ac1 = op.a[c].y + sc.wnew * un1;
          }
          const int pc = p + c * F;
          if (ov0 && ov1) {
            if (MODE != STEP_LAST) {
              __stcs(reinterpret_cast<float2*>(Dw + pc), make_float2(dd0, dd1));
              __stcs(reinterpret_cast<float2*>(Uw + pc), make_float2(un0, un1));
            }
            __stcs(reinterpret_cast<float2*>(Aw + pc), make_float2(ac0, ac1));
          } else {
            if (ov0) {
              if (MODE != STEP_LAST) Dw[pc] = dd0, Uw[pc] = un0;
              Aw[pc] = ac0;
            }
            if (ov1) {
              if (MODE != STEP_LAST) Dw[pc + 1] = dd1, Uw[pc + 1] = un1;
              Aw[pc + 1] = ac1;
            }
          }
        }
      }
      // operands of the next output row, one row ahead
      if (next_o < yb && op_row != next_o && (ov0 || ov1)) {
        ym_load_ops<FORCED>(Dr, Ar, Rr, f.irh2, so + next_o * NPX, F, ov0, ov1, op);
        op_row = next_o;
      }
      __syncwarp();  // every read of the slot refilled below is done
      if (t == 0 && j + YM_PREF <= uhi) {
        const int k = (j + YM_PREF) & (YM_RU - 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        ym_issue(&tmu, sm + k * YM_USLOT, bar + k, cx, j + YM_PREF + PAD, cc);
      }
    }
    if (!alive) {
      // wait (bounded) for this segment's copies still in flight, then stop
      if (t == 0) atomicAdd(ctl + 4, 1u);
      const unsigned long long t0 = zm_ns();
      for (int k = jfail; k <= uhi && k < jfail + YM_PREF; ++k) {  // requested, not yet consumed
        const int sl = k & (YM_RU - 1);
        while (!mbar_try(bar + sl, (phase >> sl) & 1u) && zm_ns() - t0 < 1000000000ull) {
        }
        phase ^= 1u << sl;
      }
      // the accumulator of every remaining own output is NaN
      const float nanv = __int_as_float(0x7fc00000);
      for (long long ww = w - ycount + (next_o - ya); own && ww < wend;) {
        const long long tl = ww / ny;
        const int y0 = (int)(ww - tl * ny);
        const int cnt = (int)((wend - ww) < (long long)(ny - y0) ? (wend - ww) : (long long)(ny - y0));
        const int rh = (int)(tl / ntx);
        const int x = g.off[0] - sc.shx + YM_TX * (int)(tl - (long long)rh * ntx) + 2 * i;
        for (int yy = 0; yy < cnt; ++yy)
          for (int e = 0; e < 2; ++e)
            if (ym_unknown_x(g, x + e))
              for (int c = 0; c < 2; ++c) f.acc[pidx(g, rh, c, x + e, g.off[1] + y0 + yy, 0)] = nanv;
        ww += cnt;
      }
    }
  }
}

// ---- host side ----------------------------------------------------------------
cudaError_t ym_map(const Geom& g, const float* u, unsigned char* out) {
  static_assert(sizeof(CUtensorMap) <= ZM_MAP_BYTES, "tensor map storage");
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  // the padded fields as rows (x) x rows (y) x components (2 per rhs)
  const cuuint64_t dims[3] = {(cuuint64_t)g.np[0], (cuuint64_t)g.np[1], (cuuint64_t)(2 * g.nrhs)};
  const cuuint64_t strides[2] = {(cuuint64_t)g.np[0] * sizeof(float), (cuuint64_t)g.field * sizeof(float)};
  const cuuint32_t box[3] = {YM_UX, 1, 2};
  const cuuint32_t es[3] = {1, 1, 1};
  CUtensorMap m;
  const CUresult rc = enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(u), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (rc != CUDA_SUCCESS) return cudaErrorInvalidValue;
  std::memcpy(out, &m, sizeof(m));
  return cudaSuccess;
}

void* ym_kernel(int mode, bool forced) {
  if (mode == STEP_FIRST) return forced ? (void*)step2d_o4_ym<STEP_FIRST, true> : (void*)step2d_o4_ym<STEP_FIRST, false>;
  if (mode == STEP_MID) return forced ? (void*)step2d_o4_ym<STEP_MID, true> : (void*)step2d_o4_ym<STEP_MID, false>;
  return forced ? (void*)step2d_o4_ym<STEP_LAST, true> : (void*)step2d_o4_ym<STEP_LAST, false>;
}

template <int MODE>
cudaError_t ym_launch(const cudaLaunchConfig_t& cfg, bool forced, const Geom& g, const WaveFields<float>& f,
                      const YmScalars& sc, unsigned* ctl, const CUtensorMap& tm) {
  return forced ? cudaLaunchKernelEx(&cfg, step2d_o4_ym<MODE, true>, g, f, sc, ctl, tm)
                : cudaLaunchKernelEx(&cfg, step2d_o4_ym<MODE, false>, g, f, sc, ctl, tm);
}

}  // namespace

// Plan of the 2D y-march for an order-4 FP32 context (shape slot 0 of the
// plan): tensor maps of both u buffers, the strip origin shift and the
// persistent grid.  Unusable (ok[0] = 0) on mapped grids and grids with fewer
// than 12 nodes along an axis.
ZmPlan plan_ymarch(const Geom& g, const float* u_a, const float* u_b, unsigned* ctl) {
  ZmPlan p;
  if (g.dim != 2 || g.mapped || g.n[0] < 12 || g.n[1] < 12 || g.off[0] + g.padx != 8) return p;
  int dev = 0, sms = 0, smem_max = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return p;
  }
  // x: a multiple of 4 keeps the bulk-tensor box 16-byte aligned and the node pairs even
  p.shx[0] = zm_shift(g.nu[0], YM_TX, g.hi_free[0] != 0, 4);
  p.shy[0] = 0;
  if (p.shx[0] < 0 || (int)YM_BYTES > smem_max) return p;
  for (int mode = 0; mode < 3; ++mode)
    for (int fo = 0; fo < 2; ++fo)
      if (cudaFuncSetAttribute(ym_kernel(mode, fo != 0), cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)YM_BYTES) != cudaSuccess) {
        cudaGetLastError();
        return p;
      }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ym_kernel(STEP_MID, false), 32, YM_BYTES) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return p;
  }
  if (ym_map(g, u_a, p.tmap[0][0]) != cudaSuccess || ym_map(g, u_b, p.tmap[0][1]) != cudaSuccess) {
    cudaGetLastError();
    return p;
  }
  const long long strips = (long long)((g.nu[0] + p.shx[0] + YM_TX - 1) / YM_TX) * g.nrhs;
  const long long work = strips * g.nu[1];
  // every CTA marches at least YM_MIN_ROWS rows (the +-4 row halo of a share is re-read)
  long long grid = (long long)per_sm * sms;
  const char* rows = getenv("EWH_YM_ROWS");
  const long long min_rows = (rows && atoi(rows) > 0) ? atoi(rows) : 32;
  if (grid > (work + min_rows - 1) / min_rows) grid = (work + min_rows - 1) / min_rows;
  if (grid < 1) grid = 1;
  p.grid[0] = (int)grid;
  p.ok[0] = 1;
  p.u_a = u_a;
  p.u_b = u_b;
  p.ctl = ctl;
  if (getenv("EWH_VERBOSE"))
    fprintf(stderr, "ewh: y-march plan: %lld strips (shift %d) x %d rows on %lld CTAs (%d per SM), %zu B shared\n",
            strips, p.shx[0], g.nu[1], grid, per_sm, (size_t)YM_BYTES);
  return p;
}

cudaError_t launch_ymarch(const Geom& g, const ZmPlan& p, const WaveFields<float>& f, StepMode mode,
                          const StepScalars& s, cudaStream_t st) {
  if (!p.ok[0]) return cudaErrorInvalidValue;
  const int b = f.u_cur == p.u_a ? 0 : (f.u_cur == p.u_b ? 1 : -1);
  if (b < 0) return cudaErrorInvalidValue;
  CUtensorMap tm;
  std::memcpy(&tm, p.tmap[0][b], sizeof(tm));
  YmScalars sc;
  for (int q = 0; q < 24; ++q) sc.tab12[q] = (float)(12.0 * SBP_CLOSURE[q / 6][q % 6]);
  sc.kt144 = (float)(s.kt / 144.0);
  sc.w0 = (float)s.w0;
  sc.wnew = (float)s.wnew;
  sc.fcos144 = (float)(144.0 * s.cosn);
  sc.bt12 = (float)(12.0 * 48.0 / 17.0);
  sc.shx = p.shx[0];
  zm_class_taps(sc.toff, sc.tcf);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p.grid[0]);
  cfg.blockDim = dim3(32);
  cfg.dynamicSmemBytes = YM_BYTES;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  const char* e = getenv("EWH_PDL");
  cfg.numAttrs = (e && e[0] == '0') ? 0 : 1;
  const bool forced = f.frho != nullptr;
  if (mode == STEP_FIRST) return ym_launch<STEP_FIRST>(cfg, forced, g, f, sc, p.ctl, tm);
  if (mode == STEP_MID) return ym_launch<STEP_MID>(cfg, forced, g, f, sc, p.ctl, tm);
  return ym_launch<STEP_LAST>(cfg, forced, g, f, sc, p.ctl, tm);
}

}  // namespace ewh
