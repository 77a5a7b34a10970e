// Order 4 (SBP), 3D, FP32: one fused launch per leapfrog level that marches
// along z.  It computes the level of the time-corrected explicit scheme
// (Section 4.3, eq. elastic-time-explicit-corrected) in increment form with
// the trapezoid accumulation of eq. (qoper), for the order-4 operator
//   M^{-1} K u = (1 / (rho h^2)) sum_a [ -D_a sigma_{.a} + H_a^{-1} B_a sigma_{.a} ]
// (pointwise energy density with fourth-order diagonal-norm SBP first
// derivatives D; the stresses sigma = lambda div u I + mu (grad u + grad u^T)).
//
// Each CTA owns tiles of 32 x TY unknown columns and walks them plane by
// plane.  Per plane it
//   - receives u^n (3 components) on the tile +- 4 nodes in x and y through a
//     bulk-tensor (TMA) load issued two planes ahead into a ring of 8 plane
//     buffers in shared memory, completed on one mbarrier per buffer;
//   - forms the stresses, scaled by 12 (12 D from unscaled central
//     differences or 12x closure rows), on the tile +- 2 nodes: the in-plane
//     components (xx, yy, xy, xz, yz) into a plane buffer, (xz, yz, zz) of
//     the own nodes into a ring of 8 planes;
//   - forms the in-plane part of -D sigma + H^{-1} B sigma of the own nodes
//     into a ring of 6 pending planes;
//   - and, for every output plane whose z stencil is complete, adds the z
//     part and applies the leapfrog/filter update (8-byte loads and stores of
//     node pairs; the operands of the next output plane are requested one
//     plane ahead).
// Only u^n, delta, acc, lambda, mu, 1/(rho h^2) (and f/rho) are read and only
// delta, u^{n+1} and acc written: the stresses never leave the chip.  Near
// the z sides the SBP closure rows reach up to 3 planes, so each stress plane
// is formed as soon as every u plane it reads has arrived and each output
// plane as soon as every stress plane it reads exists (the exact reach of
// each row of D); the ring depths hold for every z range of grids with at
// least 10 planes.
//
// The grid is persistent: the (rhs, tile, plane) work is split into equal
// contiguous shares, one per CTA, each a few (tile, z range) segments.
// Waits on the mbarriers are bounded (the wait limit of the context's control
// words): a CTA that gives up counts itself in ctl[4], fills the accumulator
// of its remaining outputs with NaN and returns.
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

constexpr int ZM_TX = 32;    // own nodes per tile along x
constexpr int ZM_UX = 40;    // u tile row: x from X0 - 4 (the bulk-tensor box width)
constexpr int ZM_SX = 36;    // stress tile row: x from X0 - 2
constexpr int ZM_RU = 8;     // u plane ring
constexpr int ZM_RS = 8;     // (xz, yz, zz) stress ring of the own nodes
constexpr int ZM_RP = 6;     // pending in-plane divergence ring
constexpr int ZM_PREF = 2;   // u planes requested ahead of the march



template <int TY>
struct ZmLayout {
  static constexpr int NT = 18 * (TY + 4);   // one stress-tile pair per thread
  static constexpr int UY = TY + 8;
  static constexpr int SY = TY + 4;
  static constexpr int UPLANE = UY * ZM_UX;   // one component of one u plane (floats)
  static constexpr int USLOT = 3 * UPLANE;
  static constexpr int OWN = TY * ZM_TX;
  static constexpr int SPLANE = SY * ZM_SX;   // one in-plane stress component
  static constexpr int OFF_SZ = ZM_RU * USLOT;
  static constexpr int OFF_PD = OFF_SZ + ZM_RS * 3 * OWN;
  static constexpr int OFF_SIP = OFF_PD + ZM_RP * 3 * OWN;
  static constexpr int OFF_TAB = OFF_SIP + 5 * SPLANE;
  static constexpr int OFF_CLS = OFF_TAB + 24;              // tap offsets (int) then weights, per class
  static constexpr int FLOATS = OFF_CLS + 8 * ZM_CLASSES;   // even: the mbarriers follow, 8-byte aligned
  static constexpr size_t BYTES = 128 + sizeof(float) * FLOATS + sizeof(uint64_t) * ZM_RU;
  static constexpr unsigned TX_BYTES = sizeof(float) * USLOT;  // one bulk-tensor box
  static_assert(USLOT % 32 == 0, "u ring slots stay 128-byte aligned");
  static_assert(FLOATS % 2 == 0, "mbarrier alignment");
  static_assert(OFF_CLS % 4 == 0, "16-byte table rows");
};

struct ZmScalars {
  float tab12[24];  // 12 x SBP_CLOSURE
  float kt144;      // c dt^2 / 144
  float w0, wnew;   // trapezoid weights of level 0 (first level only) and of the new level
  float fcos144;    // 144 cos(w t_n)
  float bt12;       // 12 * 48 / 17: the boundary term H^{-1} B in the scaled arithmetic
  int shx, shy;     // tile origins: off[a] - sh + tile size * k (see zm_shift)
  // 12 D at a node of class k as four taps: offsets toff[4 k ..] and weights
  // tcf[4 k ..] (classes 0..3: SBP rows 0..3 from the low side, 4: interior,
  // 5..8: rows 0..3 from the high side; zero weights pad the short rows)
  int toff[4 * ZM_CLASSES];
  float tcf[4 * ZM_CLASSES];
};

// Stresses (scaled by 12) at one node from its nine scaled derivatives
// d[c][a] = 12 D_a u_c; out: xx, yy, zz, xy, xz, yz.
__device__ __forceinline__ void zm_sigma(const float d[3][3], float l, float m, float s[6]) {
  const float div = d[0][0] + d[1][1] + d[2][2];
  const float m2 = 2.0f * m;
  s[0] = l * div + m2 * d[0][0];
  s[1] = l * div + m2 * d[1][1];
  s[2] = l * div + m2 * d[2][2];
  s[3] = m * (d[0][1] + d[1][0]);
  s[4] = m * (d[0][2] + d[2][0]);
  s[5] = m * (d[1][2] + d[2][1]);
}

struct ZmOperands {  // update operands of one own node pair at one output plane
  float2 d[3], a[3], f[3], irh;
};

// Offset of node (x, y) of plane 0 in one padded component (32 bits: a
// component holds fewer than 2^31 nodes); plane z adds z * Geom::plane.
__device__ __forceinline__ int zm_off(const Geom& g, int x, int y) {
  return g.pz * (int)g.plane + (y + PAD) * g.np[0] + x + g.padx;
}

// Update operands of the own pair at component offset o (node pair o, o + 1;
// v0, v1: which of them are unknowns); D, A, R: delta, acc and f/rho of this
// right-hand side, F the component stride.
template <bool FORCED>
__device__ __forceinline__ void zm_load_ops(const float* D, const float* A, const float* R, const float* irh2, int o,
                                            int F, bool v0, bool v1, ZmOperands& op) {
  if (v0 && v1) {  // 8-byte aligned: x - off[0] and the padded row start are even
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      op.d[c] = __ldcs(reinterpret_cast<const float2*>(D + o + c * F));
      op.a[c] = __ldcs(reinterpret_cast<const float2*>(A + o + c * F));
      if (FORCED) op.f[c] = __ldg(reinterpret_cast<const float2*>(R + o + c * F));
    }
    op.irh = __ldg(reinterpret_cast<const float2*>(irh2 + o));
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      op.d[c] = make_float2(v0 ? D[o + c * F] : 0.f, v1 ? D[o + c * F + 1] : 0.f);
      op.a[c] = make_float2(v0 ? A[o + c * F] : 0.f, v1 ? A[o + c * F + 1] : 0.f);
      if (FORCED) op.f[c] = make_float2(v0 ? R[o + c * F] : 0.f, v1 ? R[o + c * F + 1] : 0.f);
    }
    op.irh = make_float2(v0 ? irh2[o] : 0.f, v1 ? irh2[o + 1] : 0.f);
  }
}

// lambda, mu at the stress pair at component offset o (zero outside the grid;
// g0, g1: which nodes lie in it)
__device__ __forceinline__ void zm_load_lm(const float* lam, const float* mu, int o, bool g0, bool g1, float2& l,
                                           float2& m) {
  if (g0 && g1) {  // padded x even: 8-byte aligned
    l = __ldg(reinterpret_cast<const float2*>(lam + o));
    m = __ldg(reinterpret_cast<const float2*>(mu + o));
    return;
  }
  l = m = make_float2(0.f, 0.f);
  if (g0) l.x = __ldg(lam + o), m.x = __ldg(mu + o);
  if (g1) l.y = __ldg(lam + o + 1), m.y = __ldg(mu + o + 1);
}

__device__ __forceinline__ bool zm_unknown_x(const Geom& g, int x) { return x >= g.off[0] && x < g.off[0] + g.nu[0]; }
__device__ __forceinline__ bool zm_unknown_y(const Geom& g, int y) { return y >= g.off[1] && y < g.off[1] + g.nu[1]; }

// Every thread owns one pair of the stress tile (18 pairs x TY + 4 rows);
// the threads whose pair lies in the own tile also update those two nodes.
template <int TY>
constexpr int zm_threads() { return 18 * (TY + 4); }

template <int TY, int MODE, bool FORCED>
__global__ void __launch_bounds__(zm_threads<TY>(), TY <= 8 ? 2 : 1)
    step3d_o4_zm(Geom g, WaveFields<float> f, ZmScalars sc, unsigned* ctl, const __grid_constant__ CUtensorMap tmu) {
  using L = ZmLayout<TY>;
  extern __shared__ unsigned char zm_raw[];
  // 128-byte aligned base; offsetting the shared array itself (rather than an
  // integer round trip) keeps every access below in the shared address space
  float* const sm = reinterpret_cast<float*>(zm_raw + ((128u - (smem_u32(zm_raw) & 127u)) & 127u));
  uint64_t* const bar = reinterpret_cast<uint64_t*>(sm + L::FLOATS);
  float* const tab = sm + L::OFF_TAB;
  float* const sip = sm + L::OFF_SIP;
  const int t = threadIdx.x;
  int* const toff = reinterpret_cast<int*>(sm + L::OFF_CLS);
  float* const tcf = sm + L::OFF_CLS + 4 * ZM_CLASSES;
  if (t == 0) {  // static indices: the parameter arrays stay in the constant bank
#pragma unroll
    for (int k = 0; k < 24; ++k) tab[k] = sc.tab12[k];
#pragma unroll
    for (int k = 0; k < 4 * ZM_CLASSES; ++k) toff[k] = sc.toff[k], tcf[k] = sc.tcf[k];
    for (int k = 0; k < ZM_RU; ++k) mbar_init(bar + k, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  zm_pdl_wait();
  zm_pdl_trigger();
  const unsigned long long wait_ns = *reinterpret_cast<const volatile unsigned long long*>(ctl + 2);

  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const int ntx = (g.nu[0] + sc.shx + ZM_TX - 1) / ZM_TX, nty = (g.nu[1] + sc.shy + TY - 1) / TY, nz = g.nu[2];
  const long long W = (long long)ntx * nty * nz * g.nrhs;
  const long long wbeg = W * blockIdx.x / gridDim.x, wend = W * (blockIdx.x + 1) / gridDim.x;
  // this thread's stress-tile pair (nodes X0 - 2 + 2 pi, + 1; row Y0 - 2 + ri) and,
  // when it lies in the own tile, its own pair (i, r)
  const int pi = t % 18, ri = t / 18;
  const bool own = pi >= 1 && pi <= 16 && ri >= 2 && ri < TY + 2;
  const int i = pi - 1, r = ri - 2;
  const int F = (int)g.field;
  const float BT = sc.bt12;
  unsigned phase = 0;  // parity of the next completion of each u slot's mbarrier
  bool alive = true;
  long long w = wbeg;

  while (w < wend && alive) {
    // ---- segment: tile (rhs, tx, ty), output planes [za, zb)
    const long long tile = w / nz;
    const int zi = (int)(w - tile * nz);
    const int zcount = (int)((wend - w) < (long long)(nz - zi) ? (wend - w) : (long long)(nz - zi));
    w += zcount;
    const int rhs = (int)(tile / (ntx * nty));
    const int tt = (int)(tile - (long long)rhs * ntx * nty);
    const int X0 = g.off[0] - sc.shx + ZM_TX * (tt % ntx), Y0 = g.off[1] - sc.shy + TY * (tt / ntx);
    const int za = g.off[2] + zi, zb = za + zcount;
    // stress planes [slo, shi] the outputs read; u planes [ulo, uhi] those read
    const int slo = min(zm_lo(za, n2), zm_lo(zb - 1, n2)), shi = max(zm_hi(za, n2), zm_hi(zb - 1, n2));
    const int ulo = min(zm_lo(slo, n2), zm_lo(shi, n2)), uhi = max(zm_hi(slo, n2), zm_hi(shi, n2));
    const int hs0 = zm_hi(slo, n2), ho0 = zm_hi(za, n2);
    // bulk-tensor coordinates of the u box (padded x is a multiple of 4: Geom::padx)
    const int cx = X0 - 4 + g.padx, cy = Y0 - 4 + PAD, cc = 3 * rhs;
    __syncthreads();  // every read of the rings by the previous segment is done
    if (t == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      for (int k = ulo; k <= uhi && k < ulo + ZM_PREF; ++k)
        zm_issue(&tmu, sm + (k & (ZM_RU - 1)) * L::USLOT, bar + (k & (ZM_RU - 1)), cx, cy, k + g.pz, cc,
                 L::TX_BYTES);
    }
    // the stress pair of this thread and which of its nodes lie in the grid
    const int sx = X0 - 2 + 2 * pi, sy = Y0 - 2 + ri;
    const bool syin = sy >= 0 && sy < n1;
    const bool sg0 = syin && sx >= 0 && sx < n0, sg1 = syin && sx + 1 >= 0 && sx + 1 < n0;
    const int cx0 = zm_class(sx, n0), cx1 = zm_class(sx + 1, n0), cy0 = zm_class(sy, n1);
    // warps with a lane on an SBP closure row redo that axis with the class taps
    const unsigned am = __activemask();
    const bool wx = __any_sync(am, cx0 != 4 || cx1 != 4), wy = __any_sync(am, cy0 != 4);
    // own pair: nodes (ox, ox + 1), row oy
    const int ox = sx, oy = sy;
    const bool ov0 = own && zm_unknown_x(g, ox) && zm_unknown_y(g, oy);
    const bool ov1 = own && zm_unknown_x(g, ox + 1) && zm_unknown_y(g, oy);
    // component offsets of this thread's pairs at plane 0, and the state of this rhs
    const int PL = (int)g.plane;
    const int so = zm_off(g, sx, sy);
    const long long ro = (long long)rhs * 3 * g.field;
    const float* const Dr = f.delta + ro;
    const float* const Ar = f.acc + ro;
    const float* const Rr = FORCED ? f.frho + ro : nullptr;
    float* const Dw = f.delta + ro;
    float* const Aw = f.acc + ro;
    float* const Uw = f.u_next + ro;
    // lambda, mu of the next stress plane, requested one plane ahead
    float2 lm_l, lm_m;
    int lm_plane = slo;
    zm_load_lm(f.lam, f.mu, so + slo * PL, sg0, sg1, lm_l, lm_m);
    ZmOperands op;
    int op_plane = -1;
    if (ov0 || ov1) {
      zm_load_ops<FORCED>(Dr, Ar, Rr, f.irh2, so + za * PL, F, ov0, ov1, op);
      op_plane = za;
    }

    int next_s = slo, next_o = za, jfail = uhi + 1;
    bool wait_bad = false;
    for (int j = ulo; j <= uhi; ++j) {
      // ---- wait for u plane j (bounded)
      {
        const int k = j & (ZM_RU - 1);
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
        // no barrier here: the threads agree on a failed wait at the next one
        if (ok) phase ^= 1u << k;
        wait_bad = !ok;
      }
      // ---- stress planes whose u planes have all arrived
      bool any_sigma = false, failed = false;
      // the last stress plane complete at this step: every u plane its prefix of
      // stress planes reads has arrived (the prefix maximum of the reach is
      // max(hs0, hi(zs)), non-decreasing in zs)
      const int s_last = zm_last_ready(next_s, shi, hs0, j, n2);
      for (; next_s <= s_last;) {
        const int zs = next_s;
        if (lm_plane != zs) {
          zm_load_lm(f.lam, f.mu, so + zs * PL, sg0, sg1, lm_l, lm_m);
          lm_plane = zs;
        }
        const float* U0 = sm + (zs & (ZM_RU - 1)) * L::USLOT;
        const bool zin = zs >= 4 && zs <= n2 - 5;
        const int ly = ri + 2, lx = 2 + 2 * pi;  // u tile position of node sx
        float d0[3][3], d1[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          // central differences of the pair (8-byte loads; the u tile covers +- 4 around
          // the stress tile, so they stay in bounds even where a closure replaces them)
          const int o = c * L::UPLANE + ly * ZM_UX + lx;
          const float* Uc = U0 + o;
          const float2 a = ld2(Uc - 2), b = ld2(Uc), e = ld2(Uc + 2);
          d0[c][0] = c4u(a.x, a.y, b.y, e.x);
          d1[c][0] = c4u(a.y, b.x, e.x, e.y);
          const float2 m2 = ld2(Uc - 2 * ZM_UX), m1 = ld2(Uc - ZM_UX), p1 = ld2(Uc + ZM_UX), p2 = ld2(Uc + 2 * ZM_UX);
          d0[c][1] = c4u(m2.x, m1.x, p1.x, p2.x);
          d1[c][1] = c4u(m2.y, m1.y, p1.y, p2.y);
          if (zin) {  // uniform per plane
            const float2 zm2 = ld2(sm + ((zs - 2) & (ZM_RU - 1)) * L::USLOT + o);
            const float2 zm1 = ld2(sm + ((zs - 1) & (ZM_RU - 1)) * L::USLOT + o);
            const float2 zp1 = ld2(sm + ((zs + 1) & (ZM_RU - 1)) * L::USLOT + o);
            const float2 zp2 = ld2(sm + ((zs + 2) & (ZM_RU - 1)) * L::USLOT + o);
            d0[c][2] = c4u(zm2.x, zm1.x, zp1.x, zp2.x);
            d1[c][2] = c4u(zm2.y, zm1.y, zp1.y, zp2.y);
          } else {
            d0[c][2] = zm_closure12([&](int k) { return sm[((zs + k) & (ZM_RU - 1)) * L::USLOT + o]; }, zs, n2, tab);
            d1[c][2] = zm_closure12([&](int k) { return sm[((zs + k) & (ZM_RU - 1)) * L::USLOT + o + 1]; }, zs, n2,
                                    tab);
          }
        }
        // closure rows along x and y (nodes within 4 of a side): the warps that hold
        // one redo that axis for every lane with the taps of each lane's class
        if (wx) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float* Uc = U0 + c * L::UPLANE + ly * ZM_UX + lx;
            d0[c][0] = zm_d12t(Uc, 1, cx0, toff, tcf);
            d1[c][0] = zm_d12t(Uc + 1, 1, cx1, toff, tcf);
          }
        }
        if (wy) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float* Uc = U0 + c * L::UPLANE + ly * ZM_UX + lx;
            d0[c][1] = zm_d12t(Uc, ZM_UX, cy0, toff, tcf);
            d1[c][1] = zm_d12t(Uc + 1, ZM_UX, cy0, toff, tcf);
          }
        }
        float s0[6], s1[6];
        zm_sigma(d0, lm_l.x, lm_m.x, s0);
        zm_sigma(d1, lm_l.y, lm_m.y, s1);
        if (!sg0) {
#pragma unroll
          for (int k = 0; k < 6; ++k) s0[k] = 0.f;
        }
        if (!sg1) {
#pragma unroll
          for (int k = 0; k < 6; ++k) s1[k] = 0.f;
        }
        // in-plane components: xx, yy, xy, xz, yz
        const int ps = ri * ZM_SX + 2 * pi;
        st2(sip + ps, s0[0], s1[0]);
        st2(sip + L::SPLANE + ps, s0[1], s1[1]);
        st2(sip + 2 * L::SPLANE + ps, s0[3], s1[3]);
        st2(sip + 3 * L::SPLANE + ps, s0[4], s1[4]);
        st2(sip + 4 * L::SPLANE + ps, s0[5], s1[5]);
        if (own) {  // own nodes: (xz, yz, zz) into the ring
          float* SZ = sm + L::OFF_SZ + (zs & (ZM_RS - 1)) * 3 * L::OWN + r * ZM_TX + 2 * i;
          st2(SZ, s0[4], s1[4]);
          st2(SZ + L::OWN, s0[5], s1[5]);
          st2(SZ + 2 * L::OWN, s0[2], s1[2]);
        }
        if (zs + 1 <= shi) {
          zm_load_lm(f.lam, f.mu, so + (zs + 1) * PL, sg0, sg1, lm_l, lm_m);
          lm_plane = zs + 1;
        }
        if (__syncthreads_or(wait_bad)) {  // the stress plane is complete (or a wait gave up)
          failed = true;
          break;
        }
        any_sigma = true;
        if (zs >= za && zs < zb && (ov0 || ov1)) {
          // in-plane part of -D sigma + H^{-1} B sigma at the own pair: central
          // differences, then the closure rows and boundary terms of nodes within 4 of
          // a side
          float kx0[3], kx1[3], ky0[3], ky1[3];
          constexpr int CX[3] = {0, 2, 3}, CY[3] = {2, 1, 4};  // planes of sigma_{cx}, sigma_{cy}
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float* Sx = sip + CX[c] * L::SPLANE + ps;
            const float2 a = ld2(Sx - 2), b = ld2(Sx), e = ld2(Sx + 2);
            const float* Sy = sip + CY[c] * L::SPLANE + ps;
            const float2 m2 = ld2(Sy - 2 * ZM_SX), m1 = ld2(Sy - ZM_SX), p1 = ld2(Sy + ZM_SX), p2 = ld2(Sy + 2 * ZM_SX);
            kx0[c] = c4u(a.x, a.y, b.y, e.x);
            kx1[c] = c4u(a.y, b.x, e.x, e.y);
            ky0[c] = c4u(m2.x, m1.x, p1.x, p2.x);
            ky1[c] = c4u(m2.y, m1.y, p1.y, p2.y);
          }
          float k0[3], k1[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            k0[c] = -(kx0[c] + ky0[c]);
            k1[c] = -(kx1[c] + ky1[c]);
          }
          if (wx || wy) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const float* Sx = sip + CX[c] * L::SPLANE + ps;
              const float* Sy = sip + CY[c] * L::SPLANE + ps;
              if (wx) {
                kx0[c] = zm_d12t(Sx, 1, cx0, toff, tcf);
                kx1[c] = zm_d12t(Sx + 1, 1, cx1, toff, tcf);
              }
              if (wy) {
                ky0[c] = zm_d12t(Sy, ZM_SX, cy0, toff, tcf);
                ky1[c] = zm_d12t(Sy + 1, ZM_SX, cy0, toff, tcf);
              }
              // boundary terms H^{-1} B sigma on free sides (nodes on the side itself)
              float b0 = 0.f, b1 = 0.f;
              if (ox == 0) b0 -= BT * Sx[0];
              if (ox == n0 - 1) b0 += BT * Sx[0];
              if (ox + 1 == n0 - 1) b1 += BT * Sx[1];
              if (oy == 0) b0 -= BT * Sy[0], b1 -= BT * Sy[1];
              if (oy == n1 - 1) b0 += BT * Sy[0], b1 += BT * Sy[1];
              k0[c] = -(kx0[c] + ky0[c]) + b0;
              k1[c] = -(kx1[c] + ky1[c]) + b1;
            }
          }
          float* PD = sm + L::OFF_PD + (zs % ZM_RP) * 3 * L::OWN + r * ZM_TX + 2 * i;
#pragma unroll
          for (int c = 0; c < 3; ++c) st2(PD + c * L::OWN, k0[c], k1[c]);
        }
        ++next_s;
        if (next_s <= s_last) __syncthreads();  // another plane follows
      }
      if (!any_sigma && !failed) failed = __syncthreads_or(wait_bad) != 0;
      if (failed) {  // a wait gave up: every thread stops here
        alive = false;
        jfail = j;
        break;
      }
      // ---- output planes whose stress planes all exist
      const int o_last = zm_last_ready(next_o, zb - 1, ho0, next_s - 1, n2);
      for (; next_o <= o_last;) {
        const int zo = next_o;
        if (ov0 || ov1) {
          if (op_plane != zo) zm_load_ops<FORCED>(Dr, Ar, Rr, f.irh2, so + zo * PL, F, ov0, ov1, op);
          const int po = r * ZM_TX + 2 * i;
          const float* PD = sm + L::OFF_PD + (zo % ZM_RP) * 3 * L::OWN + po;
          float k0[3], k1[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float2 pd = ld2(PD + c * L::OWN);
            k0[c] = pd.x;
            k1[c] = pd.y;
          }
          if (zo >= 4 && zo <= n2 - 5) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const int o = L::OFF_SZ + c * L::OWN + po;
              const float2 m2 = ld2(sm + ((zo - 2) & (ZM_RS - 1)) * 3 * L::OWN + o);
              const float2 m1 = ld2(sm + ((zo - 1) & (ZM_RS - 1)) * 3 * L::OWN + o);
              const float2 p1 = ld2(sm + ((zo + 1) & (ZM_RS - 1)) * 3 * L::OWN + o);
              const float2 p2 = ld2(sm + ((zo + 2) & (ZM_RS - 1)) * 3 * L::OWN + o);
              k0[c] -= c4u(m2.x, m1.x, p1.x, p2.x);
              k1[c] -= c4u(m2.y, m1.y, p1.y, p2.y);
            }
          } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
#pragma unroll
              for (int e = 0; e < 2; ++e) {
                const int o = L::OFF_SZ + c * L::OWN + po + e;
                auto v = [&](int k) { return sm[((zo + k) & (ZM_RS - 1)) * 3 * L::OWN + o]; };
                float kc = -zm_closure12(v, zo, n2, tab);
                if (zo == 0) kc -= BT * v(0);
                else if (zo == n2 - 1) kc += BT * v(0);
                if (e) k1[c] += kc;
                else k0[c] += kc;
              }
            }
          }
          // leapfrog / filter update of the pair (increment form)
          const float* Uo = sm + (zo & (ZM_RU - 1)) * L::USLOT + (r + 4) * ZM_UX + 4 + 2 * i;
          const int p = so + zo * PL;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float2 u = ld2(Uo + c * L::UPLANE);
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
        ++next_o;
      }
      // operands of the next output plane, one plane ahead
      if (next_o < zb && op_plane != next_o && (ov0 || ov1)) {
        zm_load_ops<FORCED>(Dr, Ar, Rr, f.irh2, so + next_o * PL, F, ov0, ov1, op);
        op_plane = next_o;
      }
      __syncthreads();  // every read of the slot refilled below is done
      if (t == 0 && j + ZM_PREF <= uhi) {
        const int k = (j + ZM_PREF) & (ZM_RU - 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        zm_issue(&tmu, sm + k * L::USLOT, bar + k, cx, cy, j + ZM_PREF + g.pz, cc, L::TX_BYTES);
      }
    }
    if (!alive) {
      // wait (bounded) for this segment's copies still in flight, then stop
      if (t == 0) atomicAdd(ctl + 4, 1u);
      const unsigned long long t0 = zm_ns();
      for (int k = jfail; k <= uhi && k < jfail + ZM_PREF; ++k) {  // requested, not yet consumed
        const int sl = k & (ZM_RU - 1);
        while (!mbar_try(bar + sl, (phase >> sl) & 1u) && zm_ns() - t0 < 1000000000ull) {
        }
        phase ^= 1u << sl;
      }
      // the accumulator of every remaining own output is NaN
      const float nanv = __int_as_float(0x7fc00000);
      for (long long ww = w - zcount + (next_o - za); own && ww < wend;) {
        const long long tl = ww / nz;
        const int z0 = (int)(ww - tl * nz);
        const int cnt = (int)((wend - ww) < (long long)(nz - z0) ? (wend - ww) : (long long)(nz - z0));
        const int rh = (int)(tl / (ntx * nty));
        const int t2 = (int)(tl - (long long)rh * ntx * nty);
        const int x = g.off[0] - sc.shx + ZM_TX * (t2 % ntx) + 2 * i, y = g.off[1] - sc.shy + TY * (t2 / ntx) + r;
        for (int zz = 0; zz < cnt; ++zz)
          for (int e = 0; e < 2; ++e)
            if (zm_unknown_x(g, x + e) && zm_unknown_y(g, y))
              for (int c = 0; c < 3; ++c) f.acc[pidx(g, rh, c, x + e, y, g.off[2] + z0 + zz)] = nanv;
        ww += cnt;
      }
    }
  }
}

// ---- host side ----------------------------------------------------------------
template <int TY>
cudaError_t zm_map(const Geom& g, const float* u, unsigned char* out) {
  static_assert(sizeof(CUtensorMap) <= ZM_MAP_BYTES, "tensor map storage");
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t dims[4] = {(cuuint64_t)g.np[0], (cuuint64_t)g.np[1], (cuuint64_t)g.np[2],
                              (cuuint64_t)(3 * g.nrhs)};
  const cuuint64_t strides[3] = {(cuuint64_t)g.np[0] * sizeof(float), (cuuint64_t)g.plane * sizeof(float),
                                 (cuuint64_t)g.field * sizeof(float)};
  const cuuint32_t box[4] = {ZM_UX, (cuuint32_t)(TY + 8), 1, 3};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  CUtensorMap m;
  const CUresult rc = enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(u), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (rc != CUDA_SUCCESS) return cudaErrorInvalidValue;
  std::memcpy(out, &m, sizeof(m));
  return cudaSuccess;
}

template <int TY>
void* zm_kernel(int mode, bool forced) {
  if (mode == STEP_FIRST) return forced ? (void*)step3d_o4_zm<TY, STEP_FIRST, true> : (void*)step3d_o4_zm<TY, STEP_FIRST, false>;
  if (mode == STEP_MID) return forced ? (void*)step3d_o4_zm<TY, STEP_MID, true> : (void*)step3d_o4_zm<TY, STEP_MID, false>;
  return forced ? (void*)step3d_o4_zm<TY, STEP_LAST, true> : (void*)step3d_o4_zm<TY, STEP_LAST, false>;
}


template <int TY>
void plan_one(const Geom& g, const float* u_a, const float* u_b, int sms, int smem_max, ZmPlan& p, int k) {
  using L = ZmLayout<TY>;
  p.ok[k] = 0;
  // x: a multiple of 4 keeps the bulk-tensor box 16-byte aligned and the node pairs even
  p.shx[k] = zm_shift(g.nu[0], ZM_TX, g.hi_free[0] != 0, 4);
  p.shy[k] = zm_shift(g.nu[1], TY, g.hi_free[1] != 0, 1);
  if (p.shx[k] < 0 || p.shy[k] < 0 || (int)L::BYTES > smem_max) return;
  for (int mode = 0; mode < 3; ++mode)
    for (int fo = 0; fo < 2; ++fo)
      if (cudaFuncSetAttribute(zm_kernel<TY>(mode, fo != 0), cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)L::BYTES) != cudaSuccess) {
        cudaGetLastError();
        return;
      }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, zm_kernel<TY>(STEP_MID, false), L::NT, L::BYTES) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return;
  }
  if (zm_map<TY>(g, u_a, p.tmap[k][0]) != cudaSuccess || zm_map<TY>(g, u_b, p.tmap[k][1]) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  const long long tiles =
      (long long)((g.nu[0] + p.shx[k] + ZM_TX - 1) / ZM_TX) * ((g.nu[1] + p.shy[k] + TY - 1) / TY) * g.nrhs;
  const long long work = tiles * g.nu[2];
  long long grid = (long long)per_sm * sms;
  const char* cap = getenv("EWH_ZM_GRID");  // fewer CTAs: longer (tile, z range) shares per CTA
  if (cap && atoi(cap) > 0 && atoi(cap) < grid) grid = atoi(cap);
  if (grid > work) grid = work;
  p.grid[k] = (int)grid;
  p.ok[k] = 1;
  if (getenv("EWH_VERBOSE"))
    fprintf(stderr,
            "ewh: z-march plan %d (%d rows): %lld tiles (shift %d, %d) x %d planes on %lld CTAs (%d per SM), %zu B "
            "shared\n",
            k, TY, tiles, p.shx[k], p.shy[k], g.nu[2], grid, per_sm, (size_t)L::BYTES);
}

template <int TY, int MODE>
cudaError_t zm_launch(const cudaLaunchConfig_t& cfg, bool forced, const Geom& g, const WaveFields<float>& f,
                      const ZmScalars& sc, unsigned* ctl, const CUtensorMap& tm) {
  return forced ? cudaLaunchKernelEx(&cfg, step3d_o4_zm<TY, MODE, true>, g, f, sc, ctl, tm)
                : cudaLaunchKernelEx(&cfg, step3d_o4_zm<TY, MODE, false>, g, f, sc, ctl, tm);
}

}  // namespace

// Build the fused-kernel plan of a 3D order-4 FP32 context: tensor maps of
// both u buffers per shape, the persistent grids, the shared-memory opt-in.
// A shape is unusable (the per-level pair runs) when the geometry is outside
// what the kernel handles: fewer than 12 planes along z.
ZmPlan plan_zmarch(const Geom& g, const float* u_a, const float* u_b, unsigned* ctl) {
  ZmPlan p;
  if (g.dim != 3 || g.mapped || g.n[2] < 12 || g.off[0] + g.padx != 8) return p;
  int dev = 0, sms = 0, smem_max = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return p;
  }
  plan_one<16>(g, u_a, u_b, sms, smem_max, p, 0);
  plan_one<8>(g, u_a, u_b, sms, smem_max, p, 1);
  p.u_a = u_a;
  p.u_b = u_b;
  p.ctl = ctl;
  return p;
}

cudaError_t launch_zmarch(const Geom& g, const ZmPlan& p, int k, const WaveFields<float>& f, StepMode mode,
                          const StepScalars& s, cudaStream_t st) {
  if (k < 0 || k >= ZM_SHAPES || !p.ok[k]) return cudaErrorInvalidValue;
  const int b = f.u_cur == p.u_a ? 0 : (f.u_cur == p.u_b ? 1 : -1);
  if (b < 0) return cudaErrorInvalidValue;
  CUtensorMap tm;
  std::memcpy(&tm, p.tmap[k][b], sizeof(tm));
  ZmScalars sc;
  for (int q = 0; q < 24; ++q) sc.tab12[q] = (float)(12.0 * SBP_CLOSURE[q / 6][q % 6]);
  sc.kt144 = (float)(s.kt / 144.0);
  sc.w0 = (float)s.w0;
  sc.wnew = (float)s.wnew;
  sc.fcos144 = (float)(144.0 * s.cosn);
  sc.bt12 = (float)(12.0 * 48.0 / 17.0);
  sc.shx = p.shx[k];
  sc.shy = p.shy[k];
  zm_class_taps(sc.toff, sc.tcf);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p.grid[k]);
  cfg.blockDim = dim3(k == 0 ? ZmLayout<16>::NT : ZmLayout<8>::NT);
  cfg.dynamicSmemBytes = k == 0 ? ZmLayout<16>::BYTES : ZmLayout<8>::BYTES;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  const char* e = getenv("EWH_PDL");
  cfg.numAttrs = (e && e[0] == '0') ? 0 : 1;
  const bool forced = f.frho != nullptr;
  if (k == 0) {
    if (mode == STEP_FIRST) return zm_launch<16, STEP_FIRST>(cfg, forced, g, f, sc, p.ctl, tm);
    if (mode == STEP_MID) return zm_launch<16, STEP_MID>(cfg, forced, g, f, sc, p.ctl, tm);
    return zm_launch<16, STEP_LAST>(cfg, forced, g, f, sc, p.ctl, tm);
  }
  if (mode == STEP_FIRST) return zm_launch<8, STEP_FIRST>(cfg, forced, g, f, sc, p.ctl, tm);
  if (mode == STEP_MID) return zm_launch<8, STEP_MID>(cfg, forced, g, f, sc, p.ctl, tm);
  return zm_launch<8, STEP_LAST>(cfg, forced, g, f, sc, p.ctl, tm);
}

}  // namespace ewh
