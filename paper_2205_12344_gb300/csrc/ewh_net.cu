// Layers of the learned warm start (a small convolutional encoder-decoder that
// maps medium, forcing and frequency to an initial guess for the CG solve of
// M (I - S) v = M Pi 0): 3x3 convolutions as implicit GEMMs on the BF16 tensor
// cores with FP32 accumulation, their data and weight gradients, and the small
// element-wise layers.  Activations are NHWC with channel counts that are
// multiples of 16; weights are [Co][3][3][Ci].  The paper has no learned part:
// these kernels serve the precision/warm-start forms of the solver.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <string>

#include "../../include/ewh.h"
#include "ewh_internal.cuh"

namespace {

using bf16 = __nv_bfloat16;

// D (16x8 f32) += A (16x16 bf16, row) * B (16x8 bf16, col)
__device__ __forceinline__ void mma_bf16_16816(float* d, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ unsigned ld32(const bf16* p) { return *reinterpret_cast<const unsigned*>(p); }

constexpr float LEAK = 0.1f;

// ---------------------------------------------------------------------------
// Forward 3x3 convolution, zero padding, stride 1.
// CTA: 64 pixels (one image row segment) x 64 output channels, 4 warps; warp w
// owns pixels 16w..16w+15 and all 64 channels (8 mma tiles of n = 8).  The K
// loop walks (ky, kx, 16-channel chunk); each step stages a 64x16 A tile (the
// im2col gather) and a 16x64 B tile in shared memory.
// ---------------------------------------------------------------------------
constexpr int CF_PIX = 64, CF_CO = 64, CF_KS = 16, CF_LD = 24;  // LD: padded row length (bf16)

__global__ void __launch_bounds__(128) conv3x3_fwd_kernel(const bf16* __restrict__ x, const bf16* __restrict__ w,
                                                          const float* __restrict__ bias, float* __restrict__ y_pre,
                                                          bf16* __restrict__ y_act, int act, int N, int H, int W,
                                                          int Ci, int Co) {
  __shared__ __align__(16) bf16 sA[CF_PIX][CF_LD];
  __shared__ __align__(16) bf16 sB[CF_CO][CF_LD];
  const int wx_tiles = (W + CF_PIX - 1) / CF_PIX;
  const int tile = blockIdx.x;
  const int n = tile / (H * wx_tiles);
  const int rem = tile - n * H * wx_tiles;
  const int yrow = rem / wx_tiles;
  const int x0 = (rem - yrow * wx_tiles) * CF_PIX;
  const int co0 = blockIdx.y * CF_CO;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int gid = lane >> 2, tig = lane & 3;
  float acc[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
  const int nck = Ci / CF_KS;
  for (int ky = 0; ky < 3; ++ky) {
    const int yy = yrow + ky - 1;
    for (int kx = 0; kx < 3; ++kx) {
      for (int ck = 0; ck < nck; ++ck) {
        const int ci0 = ck * CF_KS;
        // A: 64 pixels x 16 channels, two 16-byte pieces per pixel
        for (int i = tid; i < CF_PIX * 2; i += 128) {
          const int p = i >> 1, half = i & 1;
          const int xx = x0 + p + kx - 1;
          uint4 v = make_uint4(0, 0, 0, 0);
          if (yy >= 0 && yy < H && xx >= 0 && xx < W && x0 + p < W)
            v = *reinterpret_cast<const uint4*>(x + (((long long)n * H + yy) * W + xx) * Ci + ci0 + half * 8);
          *reinterpret_cast<uint4*>(&sA[p][half * 8]) = v;
        }
        // B: 64 output channels x 16 input channels
        for (int i = tid; i < CF_CO * 2; i += 128) {
          const int c = i >> 1, half = i & 1;
          uint4 v = make_uint4(0, 0, 0, 0);
          if (co0 + c < Co)
            v = *reinterpret_cast<const uint4*>(w + (((long long)(co0 + c) * 3 + ky) * 3 + kx) * Ci + ci0 + half * 8);
          *reinterpret_cast<uint4*>(&sB[c][half * 8]) = v;
        }
        __syncthreads();
        unsigned a[4];
        const int r0 = warp * 16 + gid;
        a[0] = ld32(&sA[r0][tig * 2]);
        a[1] = ld32(&sA[r0 + 8][tig * 2]);
        a[2] = ld32(&sA[r0][tig * 2 + 8]);
        a[3] = ld32(&sA[r0 + 8][tig * 2 + 8]);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          unsigned b[2];
          b[0] = ld32(&sB[j * 8 + gid][tig * 2]);
          b[1] = ld32(&sB[j * 8 + gid][tig * 2 + 8]);
          mma_bf16_16816(acc[j], a, b);
        }
        __syncthreads();
      }
    }
  }
  // epilogue: bias, optional leaky ReLU; c0,c1 at row gid, c2,c3 at row gid+8
#pragma unroll
  for (int j = 0; j < 8; ++j) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int p = warp * 16 + gid + (q >= 2 ? 8 : 0);
      const int c = co0 + j * 8 + tig * 2 + (q & 1);
      const int xx = x0 + p;
      if (xx >= W || c >= Co) continue;
      float v = acc[j][q] + (bias ? bias[c] : 0.f);
      const long long o = (((long long)n * H + yrow) * W + xx) * Co + c;
      if (y_pre) y_pre[o] = v;
      if (y_act) y_act[o] = __float2bfloat16(act == 1 ? (v > 0.f ? v : LEAK * v) : v);
    }
  }
}

// weights [Co][3][3][Ci] -> flipped/transposed [Ci][3][3][Co] (for the data gradient)
__global__ void flip_transpose_kernel(const bf16* __restrict__ w, bf16* __restrict__ wt, int Ci, int Co) {
  const long long total = (long long)Co * 9 * Ci;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int ci = (int)(i % Ci);
    const int k = (int)((i / Ci) % 9);
    const int co = (int)(i / (9LL * Ci));
    const int ky = k / 3, kx = k % 3;
    wt[(((long long)ci * 3 + (2 - ky)) * 3 + (2 - kx)) * Co + co] = w[i];
  }
}

// ---------------------------------------------------------------------------
// Weight gradient: dw[co][ky][kx][ci] = sum_p dy[p][co] x[p shifted][ci].
// CTA: 64 co x 64 ci for one (ky, kx) and one chunk of pixels (split K);
// partial sums are added into the FP32 result with atomics.  A = dy^T (co x
// pixels), B = shifted x (pixels x ci), K step = 16 pixels.
// ---------------------------------------------------------------------------
constexpr int WG_PIX_CHUNK = 1024;

__global__ void __launch_bounds__(128) conv3x3_wgrad_kernel(const bf16* __restrict__ x, const bf16* __restrict__ dy,
                                                            float* __restrict__ dw, int N, int H, int W, int Ci,
                                                            int Co) {
  __shared__ __align__(16) bf16 sA[64][CF_LD];  // [co][pixel]
  __shared__ __align__(16) bf16 sB[64][CF_LD];  // [ci][pixel]
  const int k9 = blockIdx.x % 9;
  const int ky = k9 / 3, kx = k9 % 3;
  const int ci_tiles = (Ci + 63) / 64;
  const int co0 = (blockIdx.x / 9 / ci_tiles) * 64;
  const int ci0 = ((blockIdx.x / 9) % ci_tiles) * 64;
  const long long P = (long long)N * H * W;
  const long long p_begin = (long long)blockIdx.y * WG_PIX_CHUNK;
  const long long p_end = p_begin + WG_PIX_CHUNK < P ? p_begin + WG_PIX_CHUNK : P;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int gid = lane >> 2, tig = lane & 3;
  // warp tile: 16 co (rows) x 64 ci (8 n-tiles)
  float acc[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
  for (long long pb = p_begin; pb < p_end; pb += 16) {
    // stage dy[p][co0..co0+63] transposed into sA[co][p], and the shifted x
    for (int i = tid; i < 16 * 64; i += 128) {
      const int pl = i / 64, c = i % 64;
      const long long p = pb + pl;
      bf16 vdy = __float2bfloat16(0.f), vx = __float2bfloat16(0.f);
      if (p < p_end) {
        if (co0 + c < Co) vdy = dy[p * Co + co0 + c];
        const int n = (int)(p / ((long long)H * W));
        const int r = (int)(p - (long long)n * H * W);
        const int yy = r / W + ky - 1, xx = r % W + kx - 1;
        if (ci0 + c < Ci && yy >= 0 && yy < H && xx >= 0 && xx < W)
          vx = x[(((long long)n * H + yy) * W + xx) * Ci + ci0 + c];
      }
      sA[c][pl] = vdy;
      sB[c][pl] = vx;
    }
    __syncthreads();
    unsigned a[4];
    const int r0 = warp * 16 + gid;
    a[0] = ld32(&sA[r0][tig * 2]);
    a[1] = ld32(&sA[r0 + 8][tig * 2]);
    a[2] = ld32(&sA[r0][tig * 2 + 8]);
    a[3] = ld32(&sA[r0 + 8][tig * 2 + 8]);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      unsigned b[2];
      b[0] = ld32(&sB[j * 8 + gid][tig * 2]);
      b[1] = ld32(&sB[j * 8 + gid][tig * 2 + 8]);
      mma_bf16_16816(acc[j], a, b);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int co = co0 + warp * 16 + gid + (q >= 2 ? 8 : 0);
      const int ci = ci0 + j * 8 + tig * 2 + (q & 1);
      if (co < Co && ci < Ci) atomicAdd(&dw[(((long long)co * 3 + ky) * 3 + kx) * Ci + ci], acc[j][q]);
    }
}

// ---------------------------------------------------------------------------
// Element-wise layers
// ---------------------------------------------------------------------------
__global__ void bias_grad_kernel(const float* __restrict__ dy, float* __restrict__ db, long long P, int C) {
  // one block per channel; fixed-order block reduction
  __shared__ float part[256];
  const int c = blockIdx.x;
  float s = 0.f;
  for (long long p = threadIdx.x; p < P; p += 256) s += dy[p * C + c];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[c] = part[0];
}

__global__ void leaky_bwd_kernel(const float* __restrict__ pre, const float* __restrict__ dy, float* __restrict__ dx,
                                 bf16* __restrict__ dx_bf, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float g = pre[i] > 0.f ? dy[i] : LEAK * dy[i];
    if (dx) dx[i] = g;
    if (dx_bf) dx_bf[i] = __float2bfloat16(g);
  }
}

// NHWC 2x2 average pooling (bf16 in/out) and its gradient (f32)
__global__ void avgpool2_kernel(const bf16* __restrict__ x, bf16* __restrict__ y, int N, int H, int W, int C) {
  const int Ho = H / 2, Wo = W / 2;
  const long long total = (long long)N * Ho * Wo * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long q = i / C;
    const int xo = (int)(q % Wo), yo = (int)((q / Wo) % Ho), n = (int)(q / ((long long)Wo * Ho));
    const long long b = (((long long)n * H + 2 * yo) * W + 2 * xo) * C + c;
    const float s = __bfloat162float(x[b]) + __bfloat162float(x[b + C]) + __bfloat162float(x[b + (long long)W * C]) +
                    __bfloat162float(x[b + (long long)W * C + C]);
    y[i] = __float2bfloat16(0.25f * s);
  }
}
__global__ void avgpool2_bwd_kernel(const float* __restrict__ dy, float* __restrict__ dx, int N, int H, int W, int C) {
  const long long total = (long long)N * H * W * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long q = i / C;
    const int xx = (int)(q % W), yy = (int)((q / W) % H), n = (int)(q / ((long long)W * H));
    dx[i] = 0.25f * dy[(((long long)n * (H / 2) + yy / 2) * (W / 2) + xx / 2) * C + c];
  }
}
// nearest 2x upsampling of x[N,H,W,C] into channels [c_off, c_off + C) of y[N,2H,2W,Cy]
__global__ void upsample2_kernel(const bf16* __restrict__ x, bf16* __restrict__ y, int N, int H, int W, int C, int Cy,
                                 int c_off) {
  const long long total = (long long)N * 2 * H * 2 * W * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long q = i / C;
    const int xx = (int)(q % (2 * W)), yy = (int)((q / (2 * W)) % (2 * H)), n = (int)(q / (4LL * W * H));
    y[(((long long)n * 2 * H + yy) * 2 * W + xx) * Cy + c_off + c] = x[(((long long)n * H + yy / 2) * W + xx / 2) * C + c];
  }
}
// gradient of upsample2 from channels [c_off, c_off + C) of dy[N,2H,2W,Cy]
__global__ void upsample2_bwd_kernel(const float* __restrict__ dy, float* __restrict__ dx, int N, int H, int W, int C,
                                     int Cy, int c_off) {
  const long long total = (long long)N * H * W * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long q = i / C;
    const int xx = (int)(q % W), yy = (int)((q / W) % H), n = (int)(q / ((long long)W * H));
    float s = 0.f;
    for (int dyy = 0; dyy < 2; ++dyy)
      for (int dxx = 0; dxx < 2; ++dxx)
        s += dy[(((long long)n * 2 * H + 2 * yy + dyy) * 2 * W + 2 * xx + dxx) * Cy + c_off + c];
    dx[i] = s;
  }
}
// copy x[N,H,W,C] into channels [c_off, c_off + C) of y[N,H,W,Cy] (concatenation)
__global__ void copy_channels_kernel(const bf16* __restrict__ x, bf16* __restrict__ y, long long P, int C, int Cy,
                                     int c_off) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P * C; i += (long long)gridDim.x * blockDim.x)
    y[(i / C) * Cy + c_off + (i % C)] = x[i];
}
// dx[p][c] (+)= dy[p][c_off + c]  (gradient of a concatenation slice)
__global__ void slice_channels_kernel(const float* __restrict__ dy, float* __restrict__ dx, long long P, int C, int Cy,
                                      int c_off, int accumulate) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P * C; i += (long long)gridDim.x * blockDim.x) {
    const float v = dy[(i / C) * Cy + c_off + (i % C)];
    dx[i] = accumulate ? dx[i] + v : v;
  }
}
__global__ void f32_to_bf16_kernel(const float* __restrict__ a, bf16* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16(a[i]);
}
// Adam (Kingma and Ba 2015) with bias correction; also refreshes the BF16 copy
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, bf16* __restrict__ p_bf, long long n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (p_bf) p_bf[i] = __float2bfloat16(pi);
  }
}

// Per-sample scaled L2 loss on the first `cu` of `c` channels:
//   loss_s = 1/2 ||y_s - t_s||^2 / ||t_s||^2,  grad = (y - t) / (||t_s||^2 * nsamp)
// (t is FP32 [N][P][cu], y FP32 [N][P][c]); one block per sample.
__global__ void scaled_l2_kernel(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ grad,
                                 float* __restrict__ loss, long long P, int c, int cu, int nsamp) {
  __shared__ float s_tt[256], s_dd[256];
  const int n = blockIdx.x;
  const float* yn = y + (long long)n * P * c;
  const float* tn = t + (long long)n * P * cu;
  float tt = 0.f, dd = 0.f;
  for (long long i = threadIdx.x; i < P * cu; i += 256) {
    const float d = yn[(i / cu) * c + (i % cu)] - tn[i];
    tt += tn[i] * tn[i];
    dd += d * d;
  }
  s_tt[threadIdx.x] = tt;
  s_dd[threadIdx.x] = dd;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s_tt[threadIdx.x] += s_tt[threadIdx.x + o];
      s_dd[threadIdx.x] += s_dd[threadIdx.x + o];
    }
    __syncthreads();
  }
  const float inv = 1.f / fmaxf(s_tt[0], 1e-30f);
  if (threadIdx.x == 0) loss[n] = 0.5f * s_dd[0] * inv;
  float* gn = grad + (long long)n * P * c;
  for (long long i = threadIdx.x; i < P * c; i += 256) {
    const int ch = (int)(i % c);
    gn[i] = ch < cu ? (yn[i] - tn[(i / c) * cu + ch]) * inv / nsamp : 0.f;
  }
}

int egrid(long long n) {
  long long b = (n + 255) / 256;
  if (b > 4096) b = 4096;
  return (int)(b < 1 ? 1 : b);
}

ewh_status nfail(const char* msg) {
  ewh::set_global_error(msg);
  return EWH_EINVAL;
}

ewh_status launched() {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ewh::set_global_error(std::string("warm-start kernel launch failed: ") + cudaGetErrorString(e));
    return EWH_ECUDA;
  }
  return EWH_OK;
}

}  // namespace

extern "C" {

ewh_status ewh_conv3x3_fwd(const void* x, const void* w, const float* bias, float* y_pre, void* y_act, int act, int N,
                           int H, int W, int Ci, int Co, void* stream) {
  if (!x || !w || (!y_pre && !y_act) || N < 1 || H < 1 || W < 1 || Ci < 16 || Ci % 16 || Co < 8 || Co % 8)
    return nfail("ewh_conv3x3_fwd: bad arguments (Ci multiple of 16, Co multiple of 8)");
  const int wx = (W + CF_PIX - 1) / CF_PIX;
  dim3 grid((unsigned)(N * H * wx), (unsigned)((Co + CF_CO - 1) / CF_CO));
  conv3x3_fwd_kernel<<<grid, 128, 0, (cudaStream_t)stream>>>((const bf16*)x, (const bf16*)w, bias, y_pre,
                                                             (bf16*)y_act, act, N, H, W, Ci, Co);
  return launched();
}

ewh_status ewh_conv3x3_dgrad(const void* dy, const void* w, void* w_scratch, float* dx, int N, int H, int W, int Ci,
                             int Co, void* stream) {
  if (!dy || !w || !w_scratch || !dx || Ci % 16 || Co % 16 || Ci < 16 || Co < 16)
    return nfail("ewh_conv3x3_dgrad: bad arguments (Ci, Co multiples of 16)");
  cudaStream_t st = (cudaStream_t)stream;
  flip_transpose_kernel<<<egrid(9LL * Ci * Co), 256, 0, st>>>((const bf16*)w, (bf16*)w_scratch, Ci, Co);
  const int wx = (W + CF_PIX - 1) / CF_PIX;
  dim3 grid((unsigned)(N * H * wx), (unsigned)((Ci + CF_CO - 1) / CF_CO));
  conv3x3_fwd_kernel<<<grid, 128, 0, st>>>((const bf16*)dy, (const bf16*)w_scratch, nullptr, dx, nullptr, 0, N, H, W,
                                           Co, Ci);
  return launched();
}

ewh_status ewh_conv3x3_wgrad(const void* x, const void* dy, float* dw, int N, int H, int W, int Ci, int Co,
                             void* stream) {
  if (!x || !dy || !dw || Ci % 16 || Co % 16 || Ci < 16 || Co < 16)
    return nfail("ewh_conv3x3_wgrad: bad arguments (Ci, Co multiples of 16)");
  cudaStream_t st = (cudaStream_t)stream;
  cudaMemsetAsync(dw, 0, sizeof(float) * 9LL * Ci * Co, st);
  const long long P = (long long)N * H * W;
  const int ci_t = (Ci + 63) / 64, co_t = (Co + 63) / 64;
  dim3 grid((unsigned)(9 * ci_t * co_t), (unsigned)((P + WG_PIX_CHUNK - 1) / WG_PIX_CHUNK));
  conv3x3_wgrad_kernel<<<grid, 128, 0, st>>>((const bf16*)x, (const bf16*)dy, dw, N, H, W, Ci, Co);
  return launched();
}

ewh_status ewh_bias_grad(const float* dy, float* db, long long P, int C, void* stream) {
  if (!dy || !db || P < 1 || C < 1) return nfail("ewh_bias_grad: bad arguments");
  bias_grad_kernel<<<C, 256, 0, (cudaStream_t)stream>>>(dy, db, P, C);
  return launched();
}

ewh_status ewh_leaky_relu_bwd(const float* pre, const float* dy, float* dx, void* dx_bf16, long long n, void* stream) {
  if (!pre || !dy || (!dx && !dx_bf16) || n < 0) return nfail("ewh_leaky_relu_bwd: bad arguments");
  leaky_bwd_kernel<<<egrid(n), 256, 0, (cudaStream_t)stream>>>(pre, dy, dx, (bf16*)dx_bf16, n);
  return launched();
}

ewh_status ewh_avgpool2(const void* x, void* y, int N, int H, int W, int C, void* stream) {
  if (!x || !y || H % 2 || W % 2) return nfail("ewh_avgpool2: bad arguments (H, W even)");
  avgpool2_kernel<<<egrid((long long)N * H * W * C / 4), 256, 0, (cudaStream_t)stream>>>((const bf16*)x, (bf16*)y, N,
                                                                                          H, W, C);
  return launched();
}

ewh_status ewh_avgpool2_bwd(const float* dy, float* dx, int N, int H, int W, int C, void* stream) {
  if (!dy || !dx || H % 2 || W % 2) return nfail("ewh_avgpool2_bwd: bad arguments (H, W even)");
  avgpool2_bwd_kernel<<<egrid((long long)N * H * W * C), 256, 0, (cudaStream_t)stream>>>(dy, dx, N, H, W, C);
  return launched();
}

ewh_status ewh_upsample2(const void* x, void* y, int N, int H, int W, int C, int Cy, int c_off, void* stream) {
  if (!x || !y || c_off < 0 || c_off + C > Cy) return nfail("ewh_upsample2: bad arguments");
  upsample2_kernel<<<egrid(4LL * N * H * W * C), 256, 0, (cudaStream_t)stream>>>((const bf16*)x, (bf16*)y, N, H, W, C,
                                                                                  Cy, c_off);
  return launched();
}

ewh_status ewh_upsample2_bwd(const float* dy, float* dx, int N, int H, int W, int C, int Cy, int c_off, void* stream) {
  if (!dy || !dx || c_off < 0 || c_off + C > Cy) return nfail("ewh_upsample2_bwd: bad arguments");
  upsample2_bwd_kernel<<<egrid((long long)N * H * W * C), 256, 0, (cudaStream_t)stream>>>(dy, dx, N, H, W, C, Cy,
                                                                                           c_off);
  return launched();
}

ewh_status ewh_copy_channels(const void* x, void* y, long long P, int C, int Cy, int c_off, void* stream) {
  if (!x || !y || c_off < 0 || c_off + C > Cy) return nfail("ewh_copy_channels: bad arguments");
  copy_channels_kernel<<<egrid(P * C), 256, 0, (cudaStream_t)stream>>>((const bf16*)x, (bf16*)y, P, C, Cy, c_off);
  return launched();
}

ewh_status ewh_slice_channels(const float* dy, float* dx, long long P, int C, int Cy, int c_off, int accumulate,
                              void* stream) {
  if (!dy || !dx || c_off < 0 || c_off + C > Cy) return nfail("ewh_slice_channels: bad arguments");
  slice_channels_kernel<<<egrid(P * C), 256, 0, (cudaStream_t)stream>>>(dy, dx, P, C, Cy, c_off, accumulate);
  return launched();
}

ewh_status ewh_f32_to_bf16(const float* a, void* b, long long n, void* stream) {
  if (!a || !b || n < 0) return nfail("ewh_f32_to_bf16: bad arguments");
  f32_to_bf16_kernel<<<egrid(n), 256, 0, (cudaStream_t)stream>>>(a, (bf16*)b, n);
  return launched();
}

ewh_status ewh_scaled_l2_loss(const float* y, const float* t, float* grad, float* loss, long long P, int C, int Cu,
                              int N, void* stream) {
  if (!y || !t || !grad || !loss || P < 1 || Cu < 1 || Cu > C || N < 1) return nfail("ewh_scaled_l2_loss: bad arguments");
  scaled_l2_kernel<<<N, 256, 0, (cudaStream_t)stream>>>(y, t, grad, loss, P, C, Cu, N);
  return launched();
}

ewh_status ewh_adam_step(float* param, const float* grad, float* m, float* v, void* param_bf16, long long n, float lr,
                         float beta1, float beta2, float eps, int step, void* stream) {
  if (!param || !grad || !m || !v || n < 0 || step < 1) return nfail("ewh_adam_step: bad arguments");
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  adam_kernel<<<egrid(n), 256, 0, (cudaStream_t)stream>>>(param, grad, m, v, (bf16*)param_bf16, n, lr, beta1, beta2,
                                                          eps, c1, c2);
  return launched();
}

}  // extern "C"
