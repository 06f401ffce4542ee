// U-Net of the learned Poisson warm start: BF16 activations and weights,
// FP32 accumulation, training and inference on the GPU.
//
// Architecture (four levels, channels 32/64/128/256): per level two 3x3
// convolutions with ReLU, 2x2 average pooling down, 2x2 stride-2 transposed
// convolution up, skip concatenation (upsampled channels first), 1x1 head.
// Tensors are NHWC; a concatenation buffer holds [upsampled | skip] so no
// copy is made.  The input has 2 channels (rho / s, conductor mask) padded to
// 16 so that every convolution's K is a multiple of 16.
//
// 3x3 convolutions (forward and data gradient) are implicit GEMMs on the
// tensor cores (mma.sync m16n8k16 BF16 -> FP32, ldmatrix fragments, cp.async
// double-buffered tiles): M = pixels of one row segment, N = output
// channels, K = 9 taps x input channels.  The data gradient is the same
// kernel with the weights flipped in space and transposed in channels.  The
// weight gradient is a tensor-core GEMM over pixels (M = out channels,
// N = in channels per tap) accumulated with FP32 atomics.  The transposed
// convolutions, pooling, head, loss and Adam are small CUDA-core kernels.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"
#include "philox.cuh"

namespace picgb {
namespace unet {

typedef __nv_bfloat16 bf16;

constexpr int kC[4] = {32, 64, 128, 256};
constexpr int kC0 = 32;      // channels of the top level (the head's input)
constexpr int kCin0 = 16;    // padded input channels

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid) {
  const int n = valid ? 16 : 0;   // 0 bytes read: the 16 bytes are zero-filled
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(smem)),
               "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

__device__ __forceinline__ void ldsm_x4(unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3,
                                        const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3,
                                          const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma16816(float (&d)[4], unsigned a0, unsigned a1, unsigned a2,
                                         unsigned a3, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------- 3x3 conv (implicit GEMM)
struct ConvArgs {
  const bf16 *in;
  int in_cs, in_off, cin;     // channel stride / offset / count of the input
  const bf16 *w;              // [cout][9][cin]
  const float *bias;          // [cout] or null
  bf16 *out;
  int out_cs, out_off, cout;
  int B, H, W;
  int relu;
};

constexpr int kTM = 128;      // pixels per CTA (one row segment)
constexpr int kConvThreads = 256;

template <int TN, int KC>
__global__ void __launch_bounds__(kConvThreads) k_conv3x3(ConvArgs a) {
  constexpr int LDA = KC + 8;            // padded rows: conflict-free ldmatrix
  constexpr int WARPS_N = TN / 32;
  constexpr int WARPS_M = 8 / WARPS_N;
  constexpr int WTM = kTM / WARPS_M;     // pixels per warp
  constexpr int MF = WTM / 16;
  __shared__ __align__(16) bf16 As[2][kTM * LDA];
  __shared__ __align__(16) bf16 Bs[2][TN * LDA];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp / WARPS_N, wn = warp % WARPS_N;
  const int nwt = (a.W + kTM - 1) / kTM;
  const int wt = blockIdx.x % nwt;
  const int bh = blockIdx.x / nwt;       // b * H + h
  const int h = bh % a.H;
  const int w0 = wt * kTM;
  const int n0 = blockIdx.y * TN;
  const int kchunks = a.cin / KC;
  const int nk = 9 * kchunks;

  auto load = [&](int ks, int st) {
    const int tap = ks / kchunks, c0 = (ks - tap * kchunks) * KC;
    const int di = tap / 3 - 1, dj = tap % 3 - 1;
    const int hh = h + di;
    constexpr int ACH = kTM * KC / 8;    // 16-byte chunks of the A tile
    for (int q = tid; q < ACH; q += kConvThreads) {
      const int m = q / (KC / 8), cc = (q % (KC / 8)) * 8;
      const int ww = w0 + m + dj;
      const bool ok = hh >= 0 && hh < a.H && ww >= 0 && ww < a.W;
      const bf16 *src = ok ? a.in + (size_t(bh + di) * a.W + ww) * a.in_cs + a.in_off + c0 + cc : a.in;
      cp_async16(&As[st][m * LDA + cc], src, ok);
    }
    constexpr int BCH = TN * KC / 8;
    for (int q = tid; q < BCH; q += kConvThreads) {
      const int n = q / (KC / 8), cc = (q % (KC / 8)) * 8;
      const bool ok = n0 + n < a.cout;
      const bf16 *src = ok ? a.w + (size_t(n0 + n) * 9 + tap) * a.cin + c0 + cc : a.w;
      cp_async16(&Bs[st][n * LDA + cc], src, ok);
    }
    cp_async_commit();
  };

  float acc[MF][4][4];
#pragma unroll
  for (int i = 0; i < MF; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;

  load(0, 0);
  for (int ks = 0; ks < nk; ++ks) {
    const int st = ks & 1;
    cp_async_wait_all();
    __syncthreads();
    if (ks + 1 < nk) load(ks + 1, st ^ 1);
#pragma unroll
    for (int kk = 0; kk < KC; kk += 16) {
      unsigned af[MF][4];
#pragma unroll
      for (int mf = 0; mf < MF; ++mf) {
        const int row = wm * WTM + mf * 16 + (lane & 15);
        const int col = kk + (lane >> 4) * 8;
        ldsm_x4(af[mf][0], af[mf][1], af[mf][2], af[mf][3], &As[st][row * LDA + col]);
      }
#pragma unroll
      for (int np = 0; np < 2; ++np) {     // two n16 blocks per warp (32 channels)
        unsigned b0, b1, b2, b3;
        const int mi = lane >> 3;
        const int n = wn * 32 + np * 16 + (lane & 7) + ((mi >> 1) << 3);
        const int k = kk + ((mi & 1) << 3);
        ldsm_x4(b0, b1, b2, b3, &Bs[st][n * LDA + k]);
#pragma unroll
        for (int mf = 0; mf < MF; ++mf) {
          mma16816(acc[mf][np * 2 + 0], af[mf][0], af[mf][1], af[mf][2], af[mf][3], b0, b1);
          mma16816(acc[mf][np * 2 + 1], af[mf][0], af[mf][1], af[mf][2], af[mf][3], b2, b3);
        }
      }
    }
  }
  // epilogue: bias, ReLU, BF16 store (two channels per store)
#pragma unroll
  for (int mf = 0; mf < MF; ++mf) {
#pragma unroll
    for (int nf = 0; nf < 4; ++nf) {
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int m = wm * WTM + mf * 16 + (lane >> 2) + half * 8;
        const int n = n0 + wn * 32 + nf * 8 + (lane & 3) * 2;
        if (w0 + m >= a.W || n >= a.cout) continue;
        float v0 = acc[mf][nf][half * 2 + 0], v1 = acc[mf][nf][half * 2 + 1];
        if (a.bias) {
          v0 += a.bias[n];
          v1 += a.bias[n + 1];
        }
        if (a.relu) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
        }
        bf16 *dst = a.out + (size_t(bh) * a.W + w0 + m) * a.out_cs + a.out_off + n;
        *reinterpret_cast<__nv_bfloat162 *>(dst) = __floats2bfloat162_rn(v0, v1);
      }
    }
  }
}

// ---------------------------------------------------------------- 3x3 weight gradient
// dW[co][tap][ci] += sum_p dpre[p][co] * in[p + off(tap)][ci] over a group of
// rows; 32 x 32 tile of (co, ci) per CTA, 4 warps of 16 x 16.
struct WgradArgs {
  const bf16 *dpre;           // [B][H][W][cout] (contiguous)
  const bf16 *in;
  int in_cs, in_off, cin, cout;
  float *dw;                  // [cout][9][cin] FP32, accumulated
  int B, H, W;
  int rows_per_cta;
};

constexpr int kKP = 64;       // pixels per k-step

__global__ void __launch_bounds__(128) k_wgrad3x3(WgradArgs a) {
  constexpr int LD = 32 + 8;
  __shared__ __align__(16) bf16 Ds[kKP * LD];   // [pixel][co]
  __shared__ __align__(16) bf16 Xs[kKP * LD];   // [pixel][ci]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tap = blockIdx.z;
  const int di = tap / 3 - 1, dj = tap % 3 - 1;
  const int ncb = (a.cin + 31) / 32;
  const int co0 = (blockIdx.y / ncb) * 32, ci0 = (blockIdx.y % ncb) * 32;
  const int wco = (warp >> 1) * 16, wci = (warp & 1) * 16;
  float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
  const int rows = a.B * a.H;
  const int r0 = blockIdx.x * a.rows_per_cta;
  const int r1 = min(rows, r0 + a.rows_per_cta);
  for (int r = r0; r < r1; ++r) {
    const int h = r % a.H;
    for (int w0 = 0; w0 < a.W; w0 += kKP) {
      __syncthreads();
      // 64 pixels x 32 channels of each operand = 256 chunks of 16 bytes each
      for (int q = tid; q < kKP * 4; q += 128) {
        const int p = q >> 2, cc = (q & 3) * 8;
        const int w = w0 + p;
        const bool okd = w < a.W && co0 + cc < a.cout;
        cp_async16(&Ds[p * LD + cc], okd ? a.dpre + (size_t(r) * a.W + w) * a.cout + co0 + cc : a.dpre, okd);
        const int hh = h + di, ww = w + dj;
        const bool okx = w < a.W && hh >= 0 && hh < a.H && ww >= 0 && ww < a.W && ci0 + cc < a.cin;
        cp_async16(&Xs[p * LD + cc],
                   okx ? a.in + (size_t(r + di) * a.W + ww) * a.in_cs + a.in_off + ci0 + cc : a.in, okx);
      }
      cp_async_commit();
      cp_async_wait_all();
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < kKP; kk += 16) {
        const int mi = lane >> 3, rr = lane & 7;
        // A = dpre^T (rows co, k = pixel) from [pixel][co] storage
        unsigned a0, a1, a2, a3;
        {
          const int koff = (mi >> 1) << 3, moff = (mi & 1) << 3;
          ldsm_x4_t(a0, a1, a2, a3, &Ds[(kk + koff + rr) * LD + wco + moff]);
        }
        // B = in (k = pixel, n = ci) from [pixel][ci] storage
        unsigned b0, b1, b2, b3;
        {
          const int koff = (mi & 1) << 3, noff = (mi >> 1) << 3;
          ldsm_x4_t(b0, b1, b2, b3, &Xs[(kk + koff + rr) * LD + wci + noff]);
        }
        mma16816(acc[0], a0, a1, a2, a3, b0, b1);
        mma16816(acc[1], a0, a1, a2, a3, b2, b3);
      }
    }
  }
#pragma unroll
  for (int nf = 0; nf < 2; ++nf)
#pragma unroll
    for (int half = 0; half < 2; ++half)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int co = co0 + wco + (lane >> 2) + half * 8;
        const int ci = ci0 + wci + nf * 8 + (lane & 3) * 2 + e;
        if (co < a.cout && ci < a.cin)
          atomicAdd(&a.dw[(size_t(co) * 9 + tap) * a.cin + ci], acc[nf][half * 2 + e]);
      }
}

// ---------------------------------------------------------------- elementwise kernels
#define GSTRIDE(i, n) \
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)


// backward through the ReLU, with the bias gradient: dpre[p][c] = g[p][c] where
// y[p][c] > 0, else 0, and db[c] += sum_p dpre[p][c].  With POOL, g first gains
// the average pool's gradient 0.25 gp[parent of p][c] (gp [B][H/2][W/2][C]),
// rounded to BF16 as a stored sum would be.  Each thread moves 8 channels (16
// bytes) of a pixel and keeps one channel group for the whole grid-stride loop,
// so its 8 bias sums are reduced once per block.  C, channel strides and
// offsets multiples of 8.
template <bool POOL>
__global__ void __launch_bounds__(256) k_relu_back(const bf16 *g, int g_cs, int g_off, const bf16 *y, int y_cs,
                                                   int y_off, const bf16 *gp, int H, int W, bf16 *dpre, int C,
                                                   long long npix, float *db) {
  const int G = C >> 3, grp = threadIdx.x % G, ppb = blockDim.x / G;
  float s[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) s[k] = 0.f;
  for (long long p = blockIdx.x * (long long)ppb + threadIdx.x / G; p < npix; p += (long long)gridDim.x * ppb) {
    uint4 gv = *reinterpret_cast<const uint4 *>(g + p * g_cs + g_off + 8 * grp);
    const uint4 yv = *reinterpret_cast<const uint4 *>(y + p * y_cs + y_off + 8 * grp);
    bf16 *gg = reinterpret_cast<bf16 *>(&gv);
    const bf16 *yy = reinterpret_cast<const bf16 *>(&yv);
    if (POOL) {
      const int w = int(p % W);
      const long long r = p / W;   // b H + h
      const int h = int(r % H);
      const long long b = r / H;
      const uint4 pv =
          *reinterpret_cast<const uint4 *>(gp + ((b * (H / 2) + h / 2) * (W / 2) + w / 2) * C + 8 * grp);
      const bf16 *pp = reinterpret_cast<const bf16 *>(&pv);
#pragma unroll
      for (int k = 0; k < 8; ++k) gg[k] = __float2bfloat16(__bfloat162float(gg[k]) + 0.25f * __bfloat162float(pp[k]));
    }
    uint4 ov;
    bf16 *oo = reinterpret_cast<bf16 *>(&ov);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      oo[k] = __bfloat162float(yy[k]) > 0.f ? gg[k] : __float2bfloat16(0.f);
      s[k] += __bfloat162float(oo[k]);
    }
    *reinterpret_cast<uint4 *>(dpre + p * C + 8 * grp) = ov;
  }
  __shared__ float red[8][256];
#pragma unroll
  for (int k = 0; k < 8; ++k) red[k][threadIdx.x] = s[k];
  __syncthreads();
  if (int(threadIdx.x) < C) {
    const int q = threadIdx.x >> 3, k = threadIdx.x & 7;
    float t = 0.f;
    for (int j = q; j < int(blockDim.x); j += G) t += red[k][j];
    atomicAdd(&db[threadIdx.x], t);
  }
}

// W'[ci][tap][co] = W[co][8 - tap][ci]
__global__ void k_wflip(const bf16 *w, bf16 *wt, int cout, int cin) {
  GSTRIDE(i, (long long)cout * 9 * cin) {
    const int ci = int(i % cin);
    const int tap = int((i / cin) % 9);
    const int co = int(i / (9LL * cin));
    wt[(size_t(ci) * 9 + (8 - tap)) * cout + co] = w[i];
  }
}


// transposed 2x2 stride-2 convolution: out (2h x 2w) from in (h x w); W [2][2][ci][co] FP32
__global__ void k_up_fwd(const bf16 *in, int cin, const float *w, const float *bias, bf16 *out,
                         int out_cs, int out_off, int cout, int B, int h, int wd) {
  const int H = 2 * h, W = 2 * wd;
  GSTRIDE(i, (long long)B * H * W * cout) {
    const int co = int(i % cout);
    const long long p = i / cout;
    const int x = int(p % W), y = int((p / W) % H), b = int(p / ((long long)W * H));
    const int a = y & 1, c = x & 1;
    const bf16 *src = in + ((size_t(b) * h + (y >> 1)) * wd + (x >> 1)) * cin;
    const float *wk = w + (size_t(a * 2 + c) * cin) * cout + co;
    float s = bias[co];
    for (int ci = 0; ci < cin; ++ci) s = fmaf(__bfloat162float(src[ci]), wk[size_t(ci) * cout], s);
    out[p * out_cs + out_off + co] = __float2bfloat16(s);
  }
}

// data gradient of the transposed convolution: gin (h x w, cin) from gout (2h x 2w, cout)
__global__ void k_up_back_data(const bf16 *gout, int gout_cs, int gout_off, int cout, const float *w,
                               bf16 *gin, int cin, int B, int h, int wd) {
  const int W = 2 * wd;
  GSTRIDE(i, (long long)B * h * wd * cin) {
    const int ci = int(i % cin);
    const long long p = i / cin;
    const int x = int(p % wd), y = int((p / wd) % h), b = int(p / ((long long)wd * h));
    float s = 0.f;
    for (int a = 0; a < 2; ++a)
      for (int c = 0; c < 2; ++c) {
        const bf16 *g = gout + ((size_t(b) * 2 * h + 2 * y + a) * W + 2 * x + c) * gout_cs + gout_off;
        const float *wk = w + (size_t(a * 2 + c) * cin + ci) * cout;
        for (int co = 0; co < cout; ++co) s = fmaf(__bfloat162float(g[co]), wk[co], s);
      }
    gin[i] = __float2bfloat16(s);
  }
}

// weight gradient of the transposed convolution: dw[a][c][ci][co] += sum over input pixels
// of in[p][ci] * gout[child (a, c) of p][co]; one CTA per (a c, 32 ci, 32 co) and row group
__global__ void __launch_bounds__(256) k_up_back_w(const bf16 *in, int cin, const bf16 *gout,
                                                   int gout_cs, int gout_off, int cout, float *dw,
                                                   float *db, int B, int h, int wd, int rows_per_cta) {
  __shared__ float xs[32][33], gs[32][33];
  const int ac = blockIdx.z, a = ac >> 1, c = ac & 1;
  const int ncb = (cout + 31) / 32;
  const int ci0 = (blockIdx.y / ncb) * 32, co0 = (blockIdx.y % ncb) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  float bacc = 0.f;
  const int rows = B * h;
  const int r0 = blockIdx.x * rows_per_cta, r1 = min(rows, r0 + rows_per_cta);
  const int W = 2 * wd;
  for (int r = r0; r < r1; ++r) {
    const int b = r / h, y = r % h;
    for (int x0 = 0; x0 < wd; x0 += 32) {
      __syncthreads();
      for (int k = ty; k < 32; k += 8) {
        const int x = x0 + k;
        float xv = 0.f, gv = 0.f;
        if (x < wd) {
          if (ci0 + tx < cin) xv = __bfloat162float(in[((size_t(b) * h + y) * wd + x) * cin + ci0 + tx]);
          if (co0 + tx < cout)
            gv = __bfloat162float(gout[((size_t(b) * 2 * h + 2 * y + a) * W + 2 * x + c) * gout_cs + gout_off + co0 + tx]);
        }
        xs[k][tx] = xv;
        gs[k][tx] = gv;
      }
      __syncthreads();
      for (int k = 0; k < 32; ++k) {
        const float g = gs[k][tx];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = fmaf(xs[k][ty * 4 + q], g, acc[q]);
        if (ty == 0 && ci0 == 0) bacc += g;
      }
    }
  }
  for (int q = 0; q < 4; ++q) {
    const int ci = ci0 + ty * 4 + q, co = co0 + tx;
    if (ci < cin && co < cout) atomicAdd(&dw[(size_t(ac) * cin + ci) * cout + co], acc[q]);
  }
  if (ty == 0 && ci0 == 0 && co0 + tx < cout) atomicAdd(&db[co0 + tx], bacc);
}


// MSE: dy = 2 (y - t) / n, loss partial sums in FP64
__global__ void k_mse(const float *y, const float *t, float *dy, long long n, double *loss) {
  double s = 0.0;
  GSTRIDE(p, n) {
    const float d = y[p] - t[p];
    dy[p] = 2.f * d / float(n);
    s += double(d) * double(d);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s / double(n));
}

// head backward: gh[p][c] = dy[p] w[c]; dw[c] += sum_p dy h; db += sum dy
// backward through the 1x1 head y[p] = b + sum_c w[c] h[p][c]: gh[p][c] = dy[p] w[c],
// dw[c] += sum_p dy[p] h[p][c], db += sum_p dy[p].  Each thread moves 8 channels
// (16 bytes) of a pixel and keeps one channel group for the whole loop.
__global__ void __launch_bounds__(256) k_head_back(const float *dy, const bf16 *hin, const float *w, bf16 *gh,
                                                   float *dw, float *db, long long npix) {
  constexpr int G = kC0 / 8, PPB = 256 / G;
  const int grp = threadIdx.x % G;
  float wk[8], s[8], bs = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    wk[k] = w[8 * grp + k];
    s[k] = 0.f;
  }
  for (long long p = blockIdx.x * (long long)PPB + threadIdx.x / G; p < npix; p += (long long)gridDim.x * PPB) {
    const float d = dy[p];
    bs += d;
    const uint4 hv = *reinterpret_cast<const uint4 *>(hin + p * kC0 + 8 * grp);
    const bf16 *hh = reinterpret_cast<const bf16 *>(&hv);
    uint4 ov;
    bf16 *oo = reinterpret_cast<bf16 *>(&ov);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      oo[k] = __float2bfloat16(d * wk[k]);
      s[k] = fmaf(d, __bfloat162float(hh[k]), s[k]);
    }
    *reinterpret_cast<uint4 *>(gh + p * kC0 + 8 * grp) = ov;
  }
  __shared__ float red[9][256];
#pragma unroll
  for (int k = 0; k < 8; ++k) red[k][threadIdx.x] = s[k];
  red[8][threadIdx.x] = grp == 0 ? bs : 0.f;
  __syncthreads();
  if (threadIdx.x <= kC0) {
    float t = 0.f;
    if (threadIdx.x < kC0) {
      const int q = threadIdx.x >> 3, k = threadIdx.x & 7;
      for (int j = q; j < 256; j += G) t += red[k][j];
      atomicAdd(&dw[threadIdx.x], t);
    } else {
      for (int j = 0; j < 256; j += G) t += red[8][j];
      atomicAdd(db, t);
    }
  }
}

// db[c] += sum_p g[p][g_off + c] (the transposed convolution's bias gradient),
// 8 channels (16 bytes) a thread, one channel group per thread; C, g_cs and
// g_off multiples of 8, C at most 256
__global__ void __launch_bounds__(256) k_colsum(const bf16 *g, int g_cs, int g_off, int C, long long npix,
                                                float *db) {
  const int G = C >> 3, grp = threadIdx.x % G, ppb = blockDim.x / G;
  float s[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) s[k] = 0.f;
  for (long long p = blockIdx.x * (long long)ppb + threadIdx.x / G; p < npix; p += (long long)gridDim.x * ppb) {
    const uint4 v = *reinterpret_cast<const uint4 *>(g + p * g_cs + g_off + 8 * grp);
    const bf16 *vv = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] += __bfloat162float(vv[k]);
  }
  __shared__ float red[8][256];
#pragma unroll
  for (int k = 0; k < 8; ++k) red[k][threadIdx.x] = s[k];
  __syncthreads();
  if (int(threadIdx.x) < C) {
    const int q = threadIdx.x >> 3, k = threadIdx.x & 7;
    float t = 0.f;
    for (int j = q; j < int(blockDim.x); j += G) t += red[k][j];
    atomicAdd(&db[threadIdx.x], t);
  }
}

// Adam on the FP32 master parameters
__global__ void k_adam(float *p, const float *g, float *m, float *v, long long n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  GSTRIDE(i, n) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// BF16 compute copy of a conv weight from the FP32 master [co][9][ci_m],
// expanded to ci_c >= ci_m input channels with zeros
__global__ void k_w_to_bf16(const float *m, bf16 *w, int cout, int ci_m, int ci_c) {
  GSTRIDE(i, (long long)cout * 9 * ci_c) {
    const int ci = int(i % ci_c);
    const long long ct = i / ci_c;
    w[i] = __float2bfloat16(ci < ci_m ? m[ct * ci_m + ci] : 0.f);
  }
}

// gradient of an expanded conv weight folded back to the master layout
__global__ void k_w_fold(const float *gc, float *gm, int cout, int ci_m, int ci_c) {
  GSTRIDE(i, (long long)cout * 9 * ci_m) {
    const int ci = int(i % ci_m);
    const long long ct = i / ci_m;
    gm[i] += gc[ct * ci_c + ci];
  }
}

// He initialisation (He, Zhang, Ren and Sun, ICCV 2015): w ~ N(0, gain /
// fan_in) with gain 2 for layers whose output goes through a ReLU and 1 for
// the linear head.  Element e of layer `layer` draws Philox4x32-10 with
// counter (e, layer, init tag, 0) and takes the cosine half of one
// Box-Muller pair.
__global__ void k_he_init(float *w, long long n, float std, uint2 key, uint32_t layer) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const uint4 r = philox4x32_10(make_uint4(uint32_t(e), layer, kTagInit, 0u), key);
    const float rad = sqrtf(-2.0f * logf(unit24_open(r.x)));
    w[e] = std * (rad * cospif(2.0f * unit24(r.y)));
  }
}

// the transposed convolution's FP32 weights [2][2][ci][co] as the K-major
// BF16 matrix of its GEMM: row n = (2a + c) cout + co, column ci
__global__ void k_upw_to_bf16(const float *w, bf16 *wt, int cin, int cout) {
  GSTRIDE(i, 4LL * cout * cin) {
    const long long n = i / cin;
    const int ci = int(i - n * cin);
    const int ac = int(n / cout), co = int(n - (long long)ac * cout);
    wt[i] = __float2bfloat16(w[(size_t(ac) * cin + ci) * cout + co]);
  }
}

// network input: 2 channels padded to 16 with zeros, one 32-byte row per pixel
__global__ void k_to_bf16(const float *a, bf16 *b, long long n) {
  GSTRIDE(i, n) b[i] = __float2bfloat16(a[i]);
}

__global__ void k_input_vec(const float2 *x, uint4 *out, long long npix) {
  GSTRIDE(p, npix) {
    const float2 v = x[p];
    __align__(16) bf16 o[8] = {__float2bfloat16(v.x), __float2bfloat16(v.y)};
    for (int c = 2; c < 8; ++c) o[c] = __float2bfloat16(0.f);
    out[2 * p] = *reinterpret_cast<const uint4 *>(o);
    out[2 * p + 1] = make_uint4(0u, 0u, 0u, 0u);
  }
}

// First 3x3 convolution of the network (2 input channels -> kC0) on the CUDA
// cores, straight from the FP32 input pairs.  The tensor-core kernel takes K
// in blocks of 16 channels, so there it reads and multiplies 14 zero
// channels for every 2 real ones.  Here two threads form one pixel's kC0
// outputs (half each) from its 9 x 2 BF16-rounded inputs and the same BF16
// weights (w: [kC0][9][wcin], channels 0 and 1 used), in FP32 from the bias
// on, in tap order, then ReLU (if relu) and a BF16 store to out[p][kC0].
constexpr int kIn = 2;
constexpr int kHalf = kC0 / 2;
__global__ void __launch_bounds__(256) k_conv_in(const float2 *x, const bf16 *w, int wcin, const float *bias,
                                                 bf16 *out, int B, int H, int W, int relu) {
  __shared__ float4 sw[9 * kIn][kC0 / 4];   // [2 tap + c][n / 4]
  __shared__ float sb[kC0];
  for (int i = threadIdx.x; i < 9 * kIn * kC0; i += blockDim.x) {
    const int n = i % kC0, tc = i / kC0, tap = tc / kIn, c = tc - tap * kIn;
    reinterpret_cast<float *>(sw)[i] = __bfloat162float(w[(size_t(n) * 9 + tap) * wcin + c]);
  }
  for (int i = threadIdx.x; i < kC0; i += blockDim.x) sb[i] = bias ? bias[i] : 0.f;
  __syncthreads();
  // 32-bit index arithmetic (2 B H W < 2^31, checked when the network is
  // created): 64-bit division is a long instruction sequence
  const unsigned total = 2u * unsigned(B) * unsigned(H) * unsigned(W);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const unsigned p = i >> 1;
    const int half = int(i & 1u), q0 = half * (kHalf / 4);
    const unsigned r = p / unsigned(W);
    const int wq = int(p - r * unsigned(W));
    const int h = int(r % unsigned(H));
    float acc[kHalf];
#pragma unroll
    for (int n = 0; n < kHalf; ++n) acc[n] = sb[half * kHalf + n];
#pragma unroll 1
    for (int t = 0; t < 9; ++t) {
      const int dy = t / 3 - 1, dx = t - 3 * (t / 3) - 1;
      const int hh = h + dy, ww = wq + dx;
      float2 v = make_float2(0.f, 0.f);
      if (hh >= 0 && hh < H && ww >= 0 && ww < W) v = x[int(p) + dy * W + dx];
      const float v0 = __bfloat162float(__float2bfloat16(v.x));
      const float v1 = __bfloat162float(__float2bfloat16(v.y));
#pragma unroll
      for (int q = 0; q < kHalf / 4; ++q) {
        const float4 a = sw[2 * t][q0 + q], b = sw[2 * t + 1][q0 + q];
        acc[4 * q + 0] = fmaf(v1, b.x, fmaf(v0, a.x, acc[4 * q + 0]));
        acc[4 * q + 1] = fmaf(v1, b.y, fmaf(v0, a.y, acc[4 * q + 1]));
        acc[4 * q + 2] = fmaf(v1, b.z, fmaf(v0, a.z, acc[4 * q + 2]));
        acc[4 * q + 3] = fmaf(v1, b.w, fmaf(v0, a.w, acc[4 * q + 3]));
      }
    }
    uint4 *dst = reinterpret_cast<uint4 *>(out + size_t(p) * kC0 + half * kHalf);
#pragma unroll
    for (int q = 0; q < kHalf / 8; ++q) {
      __align__(16) bf16 o[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) o[k] = __float2bfloat16(relu ? fmaxf(acc[8 * q + k], 0.f) : acc[8 * q + k]);
      dst[q] = *reinterpret_cast<const uint4 *>(o);
    }
  }
}

// 2x2 average pool, 8 channels (16 bytes) per thread
__global__ void k_pool_vec(const bf16 *in, int in_cs, int in_off, bf16 *out, int C, int B, int H, int W) {
  const int Ho = H / 2, Wo = W / 2, C8 = C / 8;
  GSTRIDE(i, (long long)B * Ho * Wo * C8) {
    const int c = int(i % C8) * 8;
    const long long p = i / C8;
    const int wo = int(p % Wo), ho = int((p / Wo) % Ho), b = int(p / ((long long)Wo * Ho));
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int a = 0; a < 2; ++a)
      for (int d = 0; d < 2; ++d) {
        const uint4 v = *reinterpret_cast<const uint4 *>(
            in + ((size_t(b) * H + 2 * ho + a) * W + 2 * wo + d) * in_cs + in_off + c);
        const bf16 *e = reinterpret_cast<const bf16 *>(&v);
        for (int k = 0; k < 8; ++k) s[k] += __bfloat162float(e[k]);
      }
    __align__(16) bf16 o[8];
    for (int k = 0; k < 8; ++k) o[k] = __float2bfloat16(0.25f * s[k]);
    *reinterpret_cast<uint4 *>(out + p * C + c) = *reinterpret_cast<const uint4 *>(o);
  }
}

// head with 16-byte loads of the 32 input channels
__global__ void k_head_vec(const bf16 *hin, const float *w, const float *b, float *y, long long npix) {
  GSTRIDE(p, npix) {
    const uint4 *src = reinterpret_cast<const uint4 *>(hin + p * kC0);
    float s = b[0];
    for (int q = 0; q < kC0 / 8; ++q) {
      const uint4 v = src[q];
      const bf16 *e = reinterpret_cast<const bf16 *>(&v);
      for (int k = 0; k < 8; ++k) s = fmaf(__bfloat162float(e[k]), w[8 * q + k], s);
    }
    y[p] = s;
  }
}

inline int gridn(long long n, int t = 256) {
  long long b = (n + t - 1) / t;
  return int(b < 1 ? 1 : (b > 65535 * 8 ? 65535 * 8 : b));
}

}  // namespace unet
}  // namespace picgb

// ============================================================================
// The network
// ============================================================================
struct pic_unet {
  int B, H, W;
  int num_sms = 1;
  cudaStream_t stream = nullptr;
  std::vector<void *> allocs;
  // parameters: FP32 master (flat, in the order of the layer list), grads, Adam moments
  float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;
  long long nparam = 0;
  long long step = 0;
  double *d_loss = nullptr;
  float *y = nullptr, *dy = nullptr;     // [B][H][W]
  float *g0tmp = nullptr;                // expanded gradient of the first conv
  struct Conv {
    int cin_m, cin_c, cout;              // master / compute input channels, outputs
    long long w_off, b_off;              // offsets into P
    picgb::unet::bf16 *w, *wt;           // BF16 weights and their flipped transpose
  } conv[14];                            // enc0a..enc3b (8), dec2a..dec0b (6)
  struct Up {
    int cin, cout;
    long long w_off, b_off;
    picgb::unet::bf16 *wt;               // BF16 [4 cout][cin], row (2a + c) cout + co (tensor cores)
    picgb::unet::bf16 *wb;               // BF16 [4 cin][cout], the master order (data gradient)
  } up[3];                               // up2, up1, up0 (index = level)
  long long head_w, head_b;
  // activations (BF16 NHWC) and gradients
  picgb::unet::bf16 *x16, *a[4], *cat[3], *da[3], *dout[3], *p[4], *b3;
  picgb::unet::bf16 *gx[4], *gcat[3], *gda[3], *gdout[3], *gp[4], *gb3, *dpre[4];
  int conv_impl = 0;                     // 3x3 convolutions: 0 tcgen05 where it applies, 1 mma.sync
  int *d_err = nullptr;                  // error word of the tcgen05 kernels (a wait gave up)
};

namespace picgb {
namespace unet {
namespace {

void *ualloc(pic_unet *u, size_t bytes) {
  void *p = nullptr;
  if (cudaMalloc(&p, (bytes + 255) & ~size_t(255)) != cudaSuccess) return nullptr;
  u->allocs.push_back(p);
  return p;
}

// conv indices
enum { E0A, E0B, E1A, E1B, E2A, E2B, E3A, E3B, D2A, D2B, D1A, D1B, D0A, D0B };

int pix(const pic_unet *u, int l) { return u->B * (u->H >> l) * (u->W >> l); }

// the tcgen05 convolution when the net uses it and the shapes allow it
bool conv_tc(pic_unet *u, const bf16 *in, int in_cs, int in_off, int cin, const bf16 *w,
             const float *bias, bf16 *out, int out_cs, int out_off, int cout, int l, bool relu) {
  if (u->conv_impl != 0) return false;
  ConvTC c;
  c.in = in;
  c.in_cs = in_cs;
  c.in_off = in_off;
  c.cin = cin;
  c.w = w;
  c.bias = bias;
  c.out = out;
  c.out_cs = out_cs;
  c.out_off = out_off;
  c.cout = cout;
  c.B = u->B;
  c.H = u->H >> l;
  c.W = u->W >> l;
  c.relu = relu ? 1 : 0;
  c.err = u->d_err;
  if (!conv3x3_tc_supported(cin, cout, in_cs, in_off, out_cs, out_off, c.W)) return false;
  return conv3x3_tc(c, u->stream) == cudaSuccess;
}

void conv_fwd(pic_unet *u, int ci, const bf16 *in, int in_cs, int in_off, bf16 *out, int out_cs,
              int out_off, int l, bool relu) {
  const pic_unet::Conv &c = u->conv[ci];
  if (conv_tc(u, in, in_cs, in_off, c.cin_c, c.w, u->P + c.b_off, out, out_cs, out_off, c.cout, l, relu))
    return;
  ConvArgs a;
  a.in = in;
  a.in_cs = in_cs;
  a.in_off = in_off;
  a.cin = c.cin_c;
  a.w = c.w;
  a.bias = u->P + c.b_off;
  a.out = out;
  a.out_cs = out_cs;
  a.out_off = out_off;
  a.cout = c.cout;
  a.B = u->B;
  a.H = u->H >> l;
  a.W = u->W >> l;
  a.relu = relu ? 1 : 0;
  const int nwt = (a.W + kTM - 1) / kTM;
  if (c.cout == 32) {
    dim3 g(a.B * a.H * nwt, 1);
    if (c.cin_c == 16) k_conv3x3<32, 16><<<g, kConvThreads, 0, u->stream>>>(a);
    else k_conv3x3<32, 32><<<g, kConvThreads, 0, u->stream>>>(a);
  } else {
    dim3 g(a.B * a.H * nwt, c.cout / 64);
    k_conv3x3<64, 32><<<g, kConvThreads, 0, u->stream>>>(a);
  }
}

// data gradient: gin (cin channels) = conv(dpre, flipped weights)
void conv_back_data(pic_unet *u, int ci, const bf16 *dpre, bf16 *gin, int gin_cs, int gin_off, int l) {
  const pic_unet::Conv &c = u->conv[ci];
  k_wflip<<<gridn((long long)c.cout * 9 * c.cin_c), 256, 0, u->stream>>>(c.w, c.wt, c.cout, c.cin_c);
  if (conv_tc(u, dpre, c.cout, 0, c.cout, c.wt, nullptr, gin, gin_cs, gin_off, c.cin_c, l, false)) return;
  ConvArgs a;
  a.in = dpre;
  a.in_cs = c.cout;
  a.in_off = 0;
  a.cin = c.cout;
  a.w = c.wt;
  a.bias = nullptr;
  a.out = gin;
  a.out_cs = gin_cs;
  a.out_off = gin_off;
  a.cout = c.cin_c;
  a.B = u->B;
  a.H = u->H >> l;
  a.W = u->W >> l;
  a.relu = 0;
  const int nwt = (a.W + kTM - 1) / kTM;
  if (a.cout == 32) {
    k_conv3x3<32, 32><<<dim3(a.B * a.H * nwt, 1), kConvThreads, 0, u->stream>>>(a);
  } else {
    k_conv3x3<64, 32><<<dim3(a.B * a.H * nwt, a.cout / 64), kConvThreads, 0, u->stream>>>(a);
  }
}

// the weight gradient on the mma.sync kernel (FP32 atomics over row groups)
void wgrad_mma(int B, int H, int W, int cin, int cout, const bf16 *dpre, const bf16 *in, int in_cs, int in_off,
               float *dw, cudaStream_t s) {
  WgradArgs a;
  a.dpre = dpre;
  a.in = in;
  a.in_cs = in_cs;
  a.in_off = in_off;
  a.cin = cin;
  a.cout = cout;
  a.dw = dw;
  a.B = B;
  a.H = H;
  a.W = W;
  const int rows = B * H;
  // enough CTAs to fill the GPU: rows split so that every (co, ci, tap) tile has work
  const int tiles = ((cout + 31) / 32) * ((cin + 31) / 32) * 9;
  int groups = std::max(1, std::min(rows, 4096 / tiles));
  a.rows_per_cta = (rows + groups - 1) / groups;
  groups = (rows + a.rows_per_cta - 1) / a.rows_per_cta;
  k_wgrad3x3<<<dim3(groups, ((cout + 31) / 32) * ((cin + 31) / 32), 9), 128, 0, s>>>(a);
}

void conv_back_weights(pic_unet *u, int ci, const bf16 *dpre, const bf16 *in, int in_cs, int in_off, int l) {
  const pic_unet::Conv &c = u->conv[ci];
  const int H = u->H >> l, W = u->W >> l;
  float *dw = (c.cin_c == c.cin_m) ? u->G + c.w_off : u->g0tmp;
  if (c.cin_c != c.cin_m) cudaMemsetAsync(u->g0tmp, 0, size_t(c.cout) * 9 * c.cin_c * 4, u->stream);
  bool done = false;
  if (u->conv_impl == 0) {
    WgradTC g;
    g.dpre = dpre;
    g.in = in;
    g.in_cs = in_cs;
    g.in_off = in_off;
    g.cin = c.cin_c;
    g.cout = c.cout;
    g.dw = dw;
    g.B = u->B;
    g.H = H;
    g.W = W;
    g.err = u->d_err;
    done = conv_wgrad_tc(g, u->stream) == cudaSuccess;
  }
  if (!done) wgrad_mma(u->B, H, W, c.cin_c, c.cout, dpre, in, in_cs, in_off, dw, u->stream);
  if (c.cin_c != c.cin_m)
    k_w_fold<<<gridn((long long)c.cout * 9 * c.cin_m), 256, 0, u->stream>>>(u->g0tmp, u->G + c.w_off,
                                                                          c.cout, c.cin_m, c.cin_c);
}

// backward through relu(conv(in)) given the gradient g at its output;
// writes the gradient at its input into gin (unless gin is null)
// gp: the gradient of the average pool that follows y's block (added to g), or null
void conv_block_back(pic_unet *u, int ci, const bf16 *g, int g_cs, int g_off, const bf16 *y, int y_cs,
                     int y_off, const bf16 *in, int in_cs, int in_off, bf16 *gin, int gin_cs,
                     int gin_off, int l, const bf16 *gp = nullptr) {
  const pic_unet::Conv &c = u->conv[ci];
  const long long np = pix(u, l);
  bf16 *dpre = u->dpre[l];
  const long long ppb = 256 / (c.cout / 8);
  const int grid = int(std::min<long long>((np + ppb - 1) / ppb, 8LL * u->num_sms));
  if (gp)
    k_relu_back<true><<<grid, 256, 0, u->stream>>>(g, g_cs, g_off, y, y_cs, y_off, gp, u->H >> l, u->W >> l,
                                                   dpre, c.cout, np, u->G + c.b_off);
  else
    k_relu_back<false><<<grid, 256, 0, u->stream>>>(g, g_cs, g_off, y, y_cs, y_off, nullptr, 1, 1, dpre,
                                                    c.cout, np, u->G + c.b_off);
  conv_back_weights(u, ci, dpre, in, in_cs, in_off, l);
  if (gin) conv_back_data(u, ci, dpre, gin, gin_cs, gin_off, l);
}

void weights_to_bf16(pic_unet *u) {
  for (auto &c : u->conv)
    k_w_to_bf16<<<gridn((long long)c.cout * 9 * c.cin_c), 256, 0, u->stream>>>(u->P + c.w_off, c.w, c.cout,
                                                                             c.cin_m, c.cin_c);
  for (auto &up : u->up) {
    k_upw_to_bf16<<<gridn(4LL * up.cout * up.cin), 256, 0, u->stream>>>(u->P + up.w_off, up.wt, up.cin,
                                                                          up.cout);
    k_to_bf16<<<gridn(4LL * up.cout * up.cin), 256, 0, u->stream>>>(u->P + up.w_off, up.wb,
                                                                      4LL * up.cout * up.cin);
  }
}

// data gradient of the transposed convolution of level l on the tensor cores:
// a GEMM of the output gradient's 4 children per input pixel (K = 4 x cout)
// with the master-order weights; false where the kernel does not apply
bool up_back_tc(pic_unet *u, int l, bf16 *gin) {
  if (u->conv_impl != 0) return false;
  const pic_unet::Up &up = u->up[l];
  ConvTC c;
  c.in = u->gcat[l];
  c.in_cs = 2 * kC[l];
  c.in_off = 0;
  c.cin = up.cout;
  c.w = up.wb;
  c.bias = nullptr;
  c.out = gin;
  c.out_cs = up.cin;
  c.out_off = 0;
  c.cout = up.cin;
  c.B = u->B;
  c.H = u->H >> (l + 1);
  c.W = u->W >> (l + 1);
  c.relu = 0;
  c.err = u->d_err;
  return conv_upback_tc(c, u->stream) == cudaSuccess;
}

// weight and bias gradients of the transposed convolution of level l (input
// hin) on the tensor cores and a vector column sum; false where the kernel does
// not apply
bool up_wgrad_tc(pic_unet *u, int l, const bf16 *hin) {
  if (u->conv_impl != 0) return false;
  const pic_unet::Up &up = u->up[l];
  UpWgradTC g;
  g.in = hin;
  g.g = u->gcat[l];
  g.cin = up.cin;
  g.g_cs = 2 * kC[l];
  g.g_off = 0;
  g.cout = up.cout;
  g.dw = u->G + up.w_off;
  g.B = u->B;
  g.H = u->H >> (l + 1);
  g.W = u->W >> (l + 1);
  g.err = u->d_err;
  if (conv_upwgrad_tc(g, u->stream) != cudaSuccess) return false;
  const long long np = pix(u, l);
  const long long ppb = 256 / (up.cout / 8);
  k_colsum<<<int(std::min<long long>((np + ppb - 1) / ppb, 8LL * u->num_sms)), 256, 0, u->stream>>>(
      u->gcat[l], 2 * kC[l], 0, up.cout, np, u->G + up.b_off);
  return true;
}

// the transposed convolution of level l on the tensor cores (GEMM columns in
// launches of at most 256); false where the kernel does not apply
bool up_tc(pic_unet *u, int l, const bf16 *in, int in_cs) {
  if (u->conv_impl != 0) return false;
  const pic_unet::Up &up = u->up[l];
  ConvTC c;
  c.in = in;
  c.in_cs = in_cs;
  c.in_off = 0;
  c.cin = up.cin;
  c.w = up.wt;
  c.bias = u->P + up.b_off;
  c.out = u->cat[l];
  c.out_cs = 2 * kC[l];
  c.out_off = 0;
  c.B = u->B;
  c.H = u->H >> (l + 1);
  c.W = u->W >> (l + 1);
  c.relu = 0;
  c.err = u->d_err;
  c.up_cout = up.cout;
  const int total = 4 * up.cout, step = total > 256 ? 256 : total;
  if (!conv3x3_tc_supported(up.cin, step, in_cs, 0, c.out_cs, 0, c.W)) return false;
  for (int n0 = 0; n0 < total; n0 += step) {
    c.cout = step;
    c.n_base = n0;
    if (conv3x3_tc(c, u->stream) != cudaSuccess) return false;
  }
  return true;
}

// keep_input: also the BF16 copy of the input padded to kCin0 channels, which
// the weight gradient of the first convolution reads
void forward(pic_unet *u, const float *x, bool keep_input) {
  const int C0 = kC[0], C1 = kC[1], C2 = kC[2], C3 = kC[3];
  if (keep_input)
    k_input_vec<<<gridn(pix(u, 0)), 256, 0, u->stream>>>(reinterpret_cast<const float2 *>(x),
                                                         reinterpret_cast<uint4 *>(u->x16), pix(u, 0));
  // encoder; each level's output is written into the skip half of its concat buffer
  {
    // the first convolution on the tensor cores (K = 9 taps x 2 channels
    // packed into 32), or with the mma.sync kernels on the CUDA cores
    const pic_unet::Conv &c = u->conv[E0A];
    const float2 *x2 = reinterpret_cast<const float2 *>(x);
    if (u->conv_impl != 0 || picgb::conv_in_tc(x2, c.w, c.cin_c, u->P + c.b_off, u->a[0], u->B, u->H, u->W, 1,
                                               u->d_err, u->stream) != cudaSuccess) {
      cudaGetLastError();
      // resident CTAs (5 of 256 threads per SM) that stage the weights once each
      const int grid = std::min(gridn(2 * pix(u, 0)), 5 * u->num_sms);
      k_conv_in<<<grid, 256, 0, u->stream>>>(x2, c.w, c.cin_c, u->P + c.b_off, u->a[0], u->B, u->H, u->W, 1);
    }
  }
  conv_fwd(u, E0B, u->a[0], C0, 0, u->cat[0], 2 * C0, C0, 0, true);
  k_pool_vec<<<gridn((long long)pix(u, 1) * C0 / 8), 256, 0, u->stream>>>(u->cat[0], 2 * C0, C0, u->p[1], C0, u->B, u->H, u->W);
  conv_fwd(u, E1A, u->p[1], C0, 0, u->a[1], C1, 0, 1, true);
  conv_fwd(u, E1B, u->a[1], C1, 0, u->cat[1], 2 * C1, C1, 1, true);
  k_pool_vec<<<gridn((long long)pix(u, 2) * C1 / 8), 256, 0, u->stream>>>(u->cat[1], 2 * C1, C1, u->p[2], C1, u->B, u->H >> 1, u->W >> 1);
  conv_fwd(u, E2A, u->p[2], C1, 0, u->a[2], C2, 0, 2, true);
  conv_fwd(u, E2B, u->a[2], C2, 0, u->cat[2], 2 * C2, C2, 2, true);
  k_pool_vec<<<gridn((long long)pix(u, 3) * C2 / 8), 256, 0, u->stream>>>(u->cat[2], 2 * C2, C2, u->p[3], C2, u->B, u->H >> 2, u->W >> 2);
  conv_fwd(u, E3A, u->p[3], C2, 0, u->a[3], C3, 0, 3, true);
  conv_fwd(u, E3B, u->a[3], C3, 0, u->b3, C3, 0, 3, true);
  // decoder
  const bf16 *h = u->b3;
  int hc = C3;
  for (int l = 2; l >= 0; --l) {
    const pic_unet::Up &up = u->up[l];
    const int hl = u->H >> (l + 1), wl = u->W >> (l + 1);
    if (!up_tc(u, l, h, hc))
      k_up_fwd<<<gridn((long long)pix(u, l) * up.cout), 256, 0, u->stream>>>(
          h, hc, u->P + up.w_off, u->P + up.b_off, u->cat[l], 2 * kC[l], 0, up.cout, u->B, hl, wl);
    const int ca = (l == 2) ? D2A : (l == 1) ? D1A : D0A;
    conv_fwd(u, ca, u->cat[l], 2 * kC[l], 0, u->da[l], kC[l], 0, l, true);
    conv_fwd(u, ca + 1, u->da[l], kC[l], 0, u->dout[l], kC[l], 0, l, true);
    h = u->dout[l];
    hc = kC[l];
  }
  k_head_vec<<<gridn(pix(u, 0)), 256, 0, u->stream>>>(u->dout[0], u->P + u->head_w, u->P + u->head_b, u->y, pix(u, 0));
}

void backward(pic_unet *u) {
  const int C3 = kC[3];
  cudaMemsetAsync(u->G, 0, size_t(u->nparam) * 4, u->stream);
  k_head_back<<<int(std::min<long long>((pix(u, 0) + 63) / 64, 8LL * u->num_sms)), 256, 0, u->stream>>>(
      u->dy, u->dout[0], u->P + u->head_w, u->gdout[0], u->G + u->head_w, u->G + u->head_b, pix(u, 0));
  // decoder, from the output up
  bf16 *g = u->gdout[0];
  for (int l = 0; l <= 2; ++l) {
    const int C = kC[l];
    const int ca = (l == 2) ? D2A : (l == 1) ? D1A : D0A;
    conv_block_back(u, ca + 1, g, C, 0, u->dout[l], C, 0, u->da[l], C, 0, u->gda[l], C, 0, l);
    conv_block_back(u, ca, u->gda[l], C, 0, u->da[l], C, 0, u->cat[l], 2 * C, 0, u->gcat[l], 2 * C, 0, l);
    // transposed conv: gradient at its input (the output of level l+1) from gcat[:, 0:C]
    const pic_unet::Up &up = u->up[l];
    const int hl = u->H >> (l + 1), wl = u->W >> (l + 1);
    const bf16 *hin = (l == 2) ? u->b3 : u->dout[l + 1];
    bf16 *gin = (l == 2) ? u->gb3 : u->gdout[l + 1];
    if (!up_back_tc(u, l, gin))
      k_up_back_data<<<gridn((long long)pix(u, l + 1) * up.cin), 256, 0, u->stream>>>(
          u->gcat[l], 2 * C, 0, up.cout, u->P + up.w_off, gin, up.cin, u->B, hl, wl);
    if (!up_wgrad_tc(u, l, hin)) {
      const int rows = u->B * hl;
      const int tiles = ((up.cin + 31) / 32) * ((up.cout + 31) / 32) * 4;
      int groups = std::max(1, std::min(rows, 2048 / tiles));
      const int rpc = (rows + groups - 1) / groups;
      groups = (rows + rpc - 1) / rpc;
      k_up_back_w<<<dim3(groups, ((up.cin + 31) / 32) * ((up.cout + 31) / 32), 4), 256, 0, u->stream>>>(
          hin, up.cin, u->gcat[l], 2 * C, 0, up.cout, u->G + up.w_off, u->G + up.b_off, u->B, hl, wl, rpc);
    }
    g = gin;
  }
  // bottleneck
  conv_block_back(u, E3B, u->gb3, C3, 0, u->b3, C3, 0, u->a[3], C3, 0, u->gx[3], C3, 0, 3);
  conv_block_back(u, E3A, u->gx[3], C3, 0, u->a[3], C3, 0, u->p[3], kC[2], 0, u->gp[3], kC[2], 0, 3);
  // encoder, back down: the pool's gradient joins the skip gradient gcat[l][C:2C]
  // inside the ReLU's backward
  for (int l = 2; l >= 0; --l) {
    const int C = kC[l];
    const int ea = 2 * l;   // E0A, E1A, E2A
    conv_block_back(u, ea + 1, u->gcat[l], 2 * C, C, u->cat[l], 2 * C, C, u->a[l], C, 0, u->gx[l], C, 0, l,
                    u->gp[l + 1]);
    if (l > 0)
      conv_block_back(u, ea, u->gx[l], C, 0, u->a[l], C, 0, u->p[l], kC[l - 1], 0, u->gp[l], kC[l - 1], 0, l);
    else
      conv_block_back(u, ea, u->gx[0], C, 0, u->a[0], C, 0, u->x16, kCin0, 0, nullptr, 0, 0, 0);
  }
}

}  // namespace
}  // namespace unet
}  // namespace picgb

using namespace picgb::unet;

extern "C" {

pic_status pic_unet_create(int32_t batch, int32_t height, int32_t width, void *stream, pic_unet **out) {
  if (!out || batch < 1 || height < 16 || width < 16 || (height % 8) || (width % 8)) return PIC_EINVAL;
  if (2LL * batch * height * width >= (1LL << 31)) return PIC_EINVAL;   // 32-bit pixel indices
  pic_unet *u = new (std::nothrow) pic_unet();
  if (!u) return PIC_ENOMEM;
  u->B = batch;
  u->H = height;
  u->W = width;
  u->stream = static_cast<cudaStream_t>(stream);
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&u->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      delete u;
      return PIC_ECUDA;
    }
  }
  // parameter layout (the order of the layer list)
  long long off = 0;
  auto add_conv = [&](int idx, int cin_m, int cin_c, int cout) {
    pic_unet::Conv &c = u->conv[idx];
    c.cin_m = cin_m;
    c.cin_c = cin_c;
    c.cout = cout;
    c.w_off = off;
    off += (long long)cout * 9 * cin_m;
    c.b_off = off;
    off += cout;
  };
  int prev = 2;
  for (int l = 0; l < 4; ++l) {
    add_conv(2 * l, prev, l == 0 ? kCin0 : prev, kC[l]);
    add_conv(2 * l + 1, kC[l], kC[l], kC[l]);
    prev = kC[l];
  }
  for (int l = 2; l >= 0; --l) {
    pic_unet::Up &up = u->up[l];
    up.cin = kC[l + 1];
    up.cout = kC[l];
    up.w_off = off;
    off += 4LL * up.cin * up.cout;
    up.b_off = off;
    off += up.cout;
    const int ca = (l == 2) ? D2A : (l == 1) ? D1A : D0A;
    add_conv(ca, 2 * kC[l], 2 * kC[l], kC[l]);
    add_conv(ca + 1, kC[l], kC[l], kC[l]);
  }
  u->head_w = off;
  off += kC[0];
  u->head_b = off;
  off += 1;
  u->nparam = off;
  bool ok = true;
  auto A = [&](size_t bytes) {
    void *p = ualloc(u, bytes);
    if (!p) ok = false;
    return p;
  };
  u->P = (float *)A(off * 4);
  u->G = (float *)A(off * 4);
  u->M = (float *)A(off * 4);
  u->V = (float *)A(off * 4);
  u->d_loss = (double *)A(8);
  u->d_err = (int *)A(4);
  for (auto &c : u->conv) {
    c.w = (bf16 *)A(size_t(c.cout) * 9 * c.cin_c * 2);
    c.wt = (bf16 *)A(size_t(c.cout) * 9 * c.cin_c * 2);
  }
  for (auto &up : u->up) {
    up.wt = (bf16 *)A(4 * size_t(up.cout) * up.cin * 2);
    up.wb = (bf16 *)A(4 * size_t(up.cout) * up.cin * 2);
  }
  u->g0tmp = (float *)A(size_t(kC[0]) * 9 * kCin0 * 4);
  const size_t np0 = size_t(batch) * height * width;
  u->y = (float *)A(np0 * 4);
  u->dy = (float *)A(np0 * 4);
  u->x16 = (bf16 *)A(np0 * kCin0 * 2);
  for (int l = 0; l < 4; ++l) {
    const size_t np = np0 >> (2 * l);
    const int C = kC[l];
    u->a[l] = (bf16 *)A(np * C * 2);
    u->gx[l] = (bf16 *)A(np * C * 2);
    u->dpre[l] = (bf16 *)A(np * 2 * C * 2);
    if (l > 0) {
      u->p[l] = (bf16 *)A(np * kC[l - 1] * 2);
      u->gp[l] = (bf16 *)A(np * kC[l - 1] * 2);
    }
    if (l < 3) {
      u->cat[l] = (bf16 *)A(np * 2 * C * 2);
      u->gcat[l] = (bf16 *)A(np * 2 * C * 2);
      u->da[l] = (bf16 *)A(np * C * 2);
      u->gda[l] = (bf16 *)A(np * C * 2);
      u->dout[l] = (bf16 *)A(np * C * 2);
      u->gdout[l] = (bf16 *)A(np * C * 2);
    } else {
      u->b3 = (bf16 *)A(np * C * 2);
      u->gb3 = (bf16 *)A(np * C * 2);
    }
  }
  if (!ok) {
    pic_unet_free(u);
    return PIC_ENOMEM;
  }
  cudaMemsetAsync(u->P, 0, size_t(off) * 4, u->stream);
  cudaMemsetAsync(u->M, 0, size_t(off) * 4, u->stream);
  cudaMemsetAsync(u->V, 0, size_t(off) * 4, u->stream);
  cudaMemsetAsync(u->d_err, 0, 4, u->stream);
  if (picgb::conv3x3_tc_prepare() != cudaSuccess) u->conv_impl = 1;   // no tcgen05 kernels: mma.sync
  cudaGetLastError();
  if (cudaStreamSynchronize(u->stream) != cudaSuccess) {
    pic_unet_free(u);
    return PIC_ECUDA;
  }
  *out = u;
  return PIC_OK;
}

int64_t pic_unet_num_params(const pic_unet *u) { return u ? u->nparam : 0; }

pic_status pic_unet_set_params(pic_unet *u, const float *host) {
  if (!u || !host) return PIC_EINVAL;
  if (cudaMemcpyAsync(u->P, host, size_t(u->nparam) * 4, cudaMemcpyHostToDevice, u->stream) != cudaSuccess)
    return PIC_ECUDA;
  cudaMemsetAsync(u->M, 0, size_t(u->nparam) * 4, u->stream);
  cudaMemsetAsync(u->V, 0, size_t(u->nparam) * 4, u->stream);
  u->step = 0;
  weights_to_bf16(u);
  return cudaStreamSynchronize(u->stream) == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

pic_status pic_unet_get_params(pic_unet *u, float *host) {
  if (!u || !host) return PIC_EINVAL;
  if (cudaMemcpyAsync(host, u->P, size_t(u->nparam) * 4, cudaMemcpyDeviceToHost, u->stream) != cudaSuccess)
    return PIC_ECUDA;
  return cudaStreamSynchronize(u->stream) == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

pic_status pic_unet_forward(pic_unet *u, const float *x, float *y) {
  if (!u || !x || !y) return PIC_EINVAL;
  forward(u, x, false);
  if (cudaMemcpyAsync(y, u->y, size_t(u->B) * u->H * u->W * 4, cudaMemcpyDeviceToDevice, u->stream) != cudaSuccess)
    return PIC_ECUDA;
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

pic_status pic_unet_gradients(pic_unet *u, const float *x, const float *t, float *host_grad, double *loss) {
  if (!u || !x || !t) return PIC_EINVAL;
  forward(u, x, true);
  cudaMemsetAsync(u->d_loss, 0, 8, u->stream);
  const long long n = (long long)u->B * u->H * u->W;
  k_mse<<<std::min(1024, gridn(n)), 256, 0, u->stream>>>(u->y, t, u->dy, n, u->d_loss);
  backward(u);
  if (host_grad &&
      cudaMemcpyAsync(host_grad, u->G, size_t(u->nparam) * 4, cudaMemcpyDeviceToHost, u->stream) != cudaSuccess)
    return PIC_ECUDA;
  if (loss && cudaMemcpyAsync(loss, u->d_loss, 8, cudaMemcpyDeviceToHost, u->stream) != cudaSuccess)
    return PIC_ECUDA;
  if (cudaStreamSynchronize(u->stream) != cudaSuccess) return PIC_ECUDA;
  int err = 0;
  if (cudaMemcpy(&err, u->d_err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return PIC_ECUDA;
  if (err) return PIC_ETIMEOUT;
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

pic_status pic_unet_train_step(pic_unet *u, const float *x, const float *t, float lr, double *loss) {
  if (!u || !x || !t) return PIC_EINVAL;
  forward(u, x, true);
  cudaMemsetAsync(u->d_loss, 0, 8, u->stream);
  const long long n = (long long)u->B * u->H * u->W;
  k_mse<<<std::min(1024, gridn(n)), 256, 0, u->stream>>>(u->y, t, u->dy, n, u->d_loss);
  backward(u);
  u->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, float(u->step)), c2 = 1.f - std::pow(b2, float(u->step));
  k_adam<<<gridn(u->nparam), 256, 0, u->stream>>>(u->P, u->G, u->M, u->V, u->nparam, lr, b1, b2, 1e-8f, c1, c2);
  weights_to_bf16(u);
  if (loss && cudaMemcpyAsync(loss, u->d_loss, 8, cudaMemcpyDeviceToHost, u->stream) != cudaSuccess)
    return PIC_ECUDA;
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

pic_status pic_unet_init(pic_unet *u, uint64_t seed) {
  if (!u) return PIC_EINVAL;
  const uint2 key = make_uint2(uint32_t(seed), uint32_t(seed >> 32));
  cudaMemsetAsync(u->P, 0, size_t(u->nparam) * 4, u->stream);   // biases 0
  uint32_t layer = 0;
  for (auto &c : u->conv) {
    const long long n = (long long)c.cout * 9 * c.cin_m;
    k_he_init<<<gridn(n), 256, 0, u->stream>>>(u->P + c.w_off, n, std::sqrt(2.0f / (9.0f * c.cin_m)),
                                                key, layer++);
  }
  for (int l = 2; l >= 0; --l) {
    const pic_unet::Up &up = u->up[l];
    const long long n = 4LL * up.cin * up.cout;
    k_he_init<<<gridn(n), 256, 0, u->stream>>>(u->P + up.w_off, n, std::sqrt(2.0f / up.cin), key, layer++);
  }
  k_he_init<<<1, 256, 0, u->stream>>>(u->P + u->head_w, kC[0], std::sqrt(1.0f / kC[0]), key, layer++);
  cudaMemsetAsync(u->M, 0, size_t(u->nparam) * 4, u->stream);
  cudaMemsetAsync(u->V, 0, size_t(u->nparam) * 4, u->stream);
  u->step = 0;
  weights_to_bf16(u);
  return cudaStreamSynchronize(u->stream) == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

pic_status pic_unet_save(pic_unet *u, const char *path) {
  if (!u || !path) return PIC_EINVAL;
  std::vector<float> h(size_t(u->nparam));
  const pic_status st = pic_unet_get_params(u, h.data());
  if (st != PIC_OK) return st;
  std::FILE *f = std::fopen(path, "wb");
  if (!f) return PIC_EINVAL;
  const size_t w = std::fwrite(h.data(), 4, h.size(), f);
  return (std::fclose(f) == 0 && w == h.size()) ? PIC_OK : PIC_EINVAL;
}

pic_status pic_unet_load(pic_unet *u, const char *path) {
  if (!u || !path) return PIC_EINVAL;
  std::FILE *f = std::fopen(path, "rb");
  if (!f) return PIC_EINVAL;
  std::vector<float> h(size_t(u->nparam) + 1);
  const size_t r = std::fread(h.data(), 4, h.size(), f);
  std::fclose(f);
  if (r != size_t(u->nparam)) return PIC_EINVAL;   // too short, or longer than this network
  return pic_unet_set_params(u, h.data());
}

}  // extern "C"

namespace {
// error word of pic_conv3x3_bf16's tcgen05 kernel (a bounded wait gave up)
__device__ int g_conv_err;
}  // namespace

extern "C" {

pic_status pic_conv3x3_bf16(int32_t impl, int32_t B, int32_t H, int32_t W, const void *in, int32_t in_cs,
                            int32_t in_off, int32_t cin, const void *w, const float *bias, int32_t relu,
                            void *out, int32_t out_cs, int32_t out_off, int32_t cout, void *stream) {
  if (!in || !w || !out || B < 1 || H < 1 || W < 1 || cin < 1 || cout < 1 || in_off + cin > in_cs ||
      out_off + cout > out_cs || impl < 0 || impl > 1)
    return PIC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bf16 *bin = static_cast<const bf16 *>(in), *bw = static_cast<const bf16 *>(w);
  bf16 *bout = static_cast<bf16 *>(out);
  if (impl == 0) {
    int *err = nullptr;
    if (cudaGetSymbolAddress((void **)&err, g_conv_err) != cudaSuccess) return PIC_ECUDA;
    if (!picgb::conv3x3_tc_supported(cin, cout, in_cs, in_off, out_cs, out_off, W)) return PIC_EINVAL;
    if (cudaMemsetAsync(err, 0, 4, s) != cudaSuccess) return PIC_ECUDA;
    picgb::ConvTC c;
    c.in = bin;
    c.in_cs = in_cs;
    c.in_off = in_off;
    c.cin = cin;
    c.w = bw;
    c.bias = bias;
    c.out = bout;
    c.out_cs = out_cs;
    c.out_off = out_off;
    c.cout = cout;
    c.B = B;
    c.H = H;
    c.W = W;
    c.relu = relu ? 1 : 0;
    c.err = err;
    if (picgb::conv3x3_tc(c, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return PIC_ECUDA;
    int e = 0;
    if (cudaMemcpy(&e, err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return PIC_ECUDA;
    if (e) {
      // the wait that gave up (1 producer, 2 MMA, 3 epilogue), for pic_last_error
      picgb::note(cudaErrorTimeout, ("tcgen05 convolution wait " + std::to_string(e)).c_str());
      return PIC_ETIMEOUT;
    }
    return PIC_OK;
  }
  // the mma.sync implicit GEMM: cout 32 (cin 16 or a multiple of 32) or a multiple of 64
  ConvArgs a;
  a.in = bin;
  a.in_cs = in_cs;
  a.in_off = in_off;
  a.cin = cin;
  a.w = bw;
  a.bias = bias;
  a.out = bout;
  a.out_cs = out_cs;
  a.out_off = out_off;
  a.cout = cout;
  a.B = B;
  a.H = H;
  a.W = W;
  a.relu = relu ? 1 : 0;
  const int nwt = (W + kTM - 1) / kTM;
  if (cout == 32 && cin == 16)
    k_conv3x3<32, 16><<<dim3(B * H * nwt, 1), kConvThreads, 0, s>>>(a);
  else if (cout == 32 && cin % 32 == 0)
    k_conv3x3<32, 32><<<dim3(B * H * nwt, 1), kConvThreads, 0, s>>>(a);
  else if (cout % 64 == 0 && cin % 32 == 0)
    k_conv3x3<64, 32><<<dim3(B * H * nwt, cout / 64), kConvThreads, 0, s>>>(a);
  else
    return PIC_EINVAL;
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return PIC_ECUDA;
  return PIC_OK;
}

pic_status pic_conv3x3_wgrad_bf16(int32_t impl, int32_t B, int32_t H, int32_t W, const void *dpre,
                                  const void *in, int32_t in_cs, int32_t in_off, int32_t cin, int32_t cout,
                                  float *dw, void *stream) {
  if (!dpre || !in || !dw || B < 1 || H < 1 || W < 1 || cin < 1 || cout < 1 || in_off < 0 ||
      in_off + cin > in_cs || impl < 0 || impl > 1 || (long long)B * H * W >= (1LL << 31))
    return PIC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bf16 *bd = static_cast<const bf16 *>(dpre), *bi = static_cast<const bf16 *>(in);
  if (impl == 1) {
    if (in_cs % 8 || in_off % 8 || cin % 8 || cout % 8) return PIC_EINVAL;   // 16-byte cp.async rows
    wgrad_mma(B, H, W, cin, cout, bd, bi, in_cs, in_off, dw, s);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return PIC_ECUDA;
    return PIC_OK;
  }
  if (!picgb::conv_wgrad_tc_supported(cin, cout, in_cs, in_off, dw)) return PIC_EINVAL;
  int *err = nullptr;
  if (cudaGetSymbolAddress((void **)&err, g_conv_err) != cudaSuccess) return PIC_ECUDA;
  if (cudaMemsetAsync(err, 0, 4, s) != cudaSuccess) return PIC_ECUDA;
  picgb::WgradTC g;
  g.dpre = bd;
  g.in = bi;
  g.in_cs = in_cs;
  g.in_off = in_off;
  g.cin = cin;
  g.cout = cout;
  g.dw = dw;
  g.B = B;
  g.H = H;
  g.W = W;
  g.err = err;
  if (picgb::conv_wgrad_tc(g, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return PIC_ECUDA;
  int e = 0;
  if (cudaMemcpy(&e, err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return PIC_ECUDA;
  if (e) {
    picgb::note(cudaErrorTimeout, ("tcgen05 weight gradient wait " + std::to_string(e)).c_str());
    return PIC_ETIMEOUT;
  }
  return PIC_OK;
}

namespace {
int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return sms;
}
bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
}  // namespace

pic_status pic_avgpool2_bf16(int32_t B, int32_t H, int32_t W, const void *in, int32_t in_cs, int32_t in_off,
                             int32_t C, void *out, void *stream) {
  if (!in || !out || B < 1 || H < 2 || W < 2 || (H % 2) || (W % 2) || C < 8 || C % 8 || in_cs % 8 ||
      in_off % 8 || in_off < 0 || in_off + C > in_cs || !aligned16(in) || !aligned16(out) ||
      (long long)B * H * W >= (1LL << 31))
    return PIC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_pool_vec<<<gridn((long long)B * (H / 2) * (W / 2) * (C / 8)), 256, 0, s>>>(
      static_cast<const bf16 *>(in), in_cs, in_off, static_cast<bf16 *>(out), C, B, H, W);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return PIC_ECUDA;
  return PIC_OK;
}

pic_status pic_head_bf16(int64_t npix, const void *hin, const float *w, const float *b, float *y, void *stream) {
  if (!hin || !w || !b || !y || npix < 1 || !aligned16(hin)) return PIC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_head_vec<<<gridn(npix), 256, 0, s>>>(static_cast<const bf16 *>(hin), w, b, y, npix);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return PIC_ECUDA;
  return PIC_OK;
}

pic_status pic_head_back_bf16(int64_t npix, const float *dy, const void *hin, const float *w, void *gh, float *dw,
                              float *db, void *stream) {
  if (!dy || !hin || !w || !gh || !dw || !db || npix < 1 || !aligned16(hin) || !aligned16(gh)) return PIC_EINVAL;
  const int sms = device_sms();
  if (sms < 1) return PIC_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_head_back<<<int(std::min<long long>((npix + 63) / 64, 8LL * sms)), 256, 0, s>>>(
      dy, static_cast<const bf16 *>(hin), w, static_cast<bf16 *>(gh), dw, db, npix);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return PIC_ECUDA;
  return PIC_OK;
}

pic_status pic_relu_back_bf16(int32_t B, int32_t H, int32_t W, const void *g, int32_t g_cs, int32_t g_off,
                              const void *y, int32_t y_cs, int32_t y_off, const void *gp, void *dpre, int32_t C,
                              float *db, void *stream) {
  if (!g || !y || !dpre || !db || B < 1 || H < 1 || W < 1 || !(C == 8 || C == 16 || C == 32 || C == 64 ||
      C == 128 || C == 256) || g_cs % 8 || g_off % 8 || y_cs % 8 || y_off % 8 || g_off < 0 || y_off < 0 ||
      g_off + C > g_cs || y_off + C > y_cs || !aligned16(g) || !aligned16(y) || !aligned16(dpre) ||
      (gp && (!aligned16(gp) || (H % 2) || (W % 2))) || (long long)B * H * W >= (1LL << 31))
    return PIC_EINVAL;
  const int sms = device_sms();
  if (sms < 1) return PIC_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long np = (long long)B * H * W, ppb = 256 / (C / 8);
  const int grid = int(std::min<long long>((np + ppb - 1) / ppb, 8LL * sms));
  const bf16 *bg = static_cast<const bf16 *>(g), *by = static_cast<const bf16 *>(y);
  if (gp)
    k_relu_back<true><<<grid, 256, 0, s>>>(bg, g_cs, g_off, by, y_cs, y_off, static_cast<const bf16 *>(gp), H, W,
                                           static_cast<bf16 *>(dpre), C, np, db);
  else
    k_relu_back<false><<<grid, 256, 0, s>>>(bg, g_cs, g_off, by, y_cs, y_off, nullptr, 1, 1,
                                            static_cast<bf16 *>(dpre), C, np, db);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return PIC_ECUDA;
  return PIC_OK;
}

pic_status pic_upconv_bf16(int32_t impl, int32_t B, int32_t H, int32_t W, const void *in, int32_t cin,
                           const float *w, const float *bias, void *out, int32_t out_cs, int32_t out_off,
                           int32_t cout, void *stream) {
  if (!in || !w || !bias || !out || B < 1 || H < 1 || W < 1 || cin < 1 || cout < 1 || out_off < 0 ||
      out_off + cout > out_cs || impl < 0 || impl > 1 || (long long)B * H * W * 4 >= (1LL << 31))
    return PIC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bf16 *bi = static_cast<const bf16 *>(in);
  bf16 *bo = static_cast<bf16 *>(out);
  if (impl == 1) {
    k_up_fwd<<<gridn(4LL * B * H * W * cout), 256, 0, s>>>(bi, cin, w, bias, bo, out_cs, out_off, cout, B, H, W);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return PIC_ECUDA;
    return PIC_OK;
  }
  const int total = 4 * cout, step = total > 256 ? 256 : total;
  if (total % step || cout % 16 || !picgb::conv3x3_tc_supported(cin, step, cin, 0, out_cs, out_off, W))
    return PIC_EINVAL;
  int *err = nullptr;
  if (cudaGetSymbolAddress((void **)&err, g_conv_err) != cudaSuccess) return PIC_ECUDA;
  bf16 *wt = nullptr;
  if (cudaMalloc(&wt, size_t(total) * cin * 2) != cudaSuccess) return PIC_ENOMEM;
  k_upw_to_bf16<<<gridn(4LL * cout * cin), 256, 0, s>>>(w, wt, cin, cout);
  picgb::ConvTC c;
  c.in = bi;
  c.in_cs = cin;
  c.in_off = 0;
  c.cin = cin;
  c.w = wt;
  c.bias = bias;
  c.out = bo;
  c.out_cs = out_cs;
  c.out_off = out_off;
  c.B = B;
  c.H = H;
  c.W = W;
  c.relu = 0;
  c.err = err;
  c.up_cout = cout;
  pic_status st = (cudaGetLastError() == cudaSuccess && cudaMemsetAsync(err, 0, 4, s) == cudaSuccess) ? PIC_OK
                                                                                                   : PIC_ECUDA;
  for (int n0 = 0; st == PIC_OK && n0 < total; n0 += step) {
    c.cout = step;
    c.n_base = n0;
    if (picgb::conv3x3_tc(c, s) != cudaSuccess) st = PIC_ECUDA;
  }
  if (st == PIC_OK && cudaStreamSynchronize(s) != cudaSuccess) st = PIC_ECUDA;
  int e = 0;
  if (st == PIC_OK && cudaMemcpy(&e, err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) st = PIC_ECUDA;
  cudaStreamSynchronize(s);
  cudaFree(wt);
  if (st == PIC_OK && e) {
    picgb::note(cudaErrorTimeout, ("tcgen05 convolution wait " + std::to_string(e)).c_str());
    st = PIC_ETIMEOUT;
  }
  return st;
}

pic_status pic_upconv_wgrad_bf16(int32_t impl, int32_t B, int32_t H, int32_t W, const void *in, int32_t cin,
                                 const void *gout, int32_t gout_cs, int32_t gout_off, int32_t cout, float *dw,
                                 float *db, void *stream) {
  if (!in || !gout || !dw || !db || B < 1 || H < 1 || W < 1 || cin < 1 || cout < 1 || gout_off < 0 ||
      gout_off + cout > gout_cs || impl < 0 || impl > 1 || (long long)B * H * W * 4 >= (1LL << 31))
    return PIC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bf16 *bi = static_cast<const bf16 *>(in), *bg = static_cast<const bf16 *>(gout);
  if (impl == 1) {
    const int rows = B * H;
    const int tiles = ((cin + 31) / 32) * ((cout + 31) / 32) * 4;
    int groups = std::max(1, std::min(rows, 2048 / tiles));
    const int rpc = (rows + groups - 1) / groups;
    groups = (rows + rpc - 1) / rpc;
    k_up_back_w<<<dim3(groups, ((cin + 31) / 32) * ((cout + 31) / 32), 4), 256, 0, s>>>(
        bi, cin, bg, gout_cs, gout_off, cout, dw, db, B, H, W, rpc);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return PIC_ECUDA;
    return PIC_OK;
  }
  if (!picgb::conv_upwgrad_tc_supported(cin, cout, gout_cs, gout_off) || cout > 256 ||
      (reinterpret_cast<uintptr_t>(gout) & 15))
    return PIC_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PIC_ECUDA;
  int *err = nullptr;
  if (cudaGetSymbolAddress((void **)&err, g_conv_err) != cudaSuccess) return PIC_ECUDA;
  if (cudaMemsetAsync(err, 0, 4, s) != cudaSuccess) return PIC_ECUDA;
  picgb::UpWgradTC g;
  g.in = bi;
  g.g = bg;
  g.cin = cin;
  g.g_cs = gout_cs;
  g.g_off = gout_off;
  g.cout = cout;
  g.dw = dw;
  g.B = B;
  g.H = H;
  g.W = W;
  g.err = err;
  if (picgb::conv_upwgrad_tc(g, s) != cudaSuccess) return PIC_ECUDA;
  const long long np = 4LL * B * H * W, ppb = 256 / (cout / 8);
  k_colsum<<<int(std::min<long long>((np + ppb - 1) / ppb, 8LL * sms)), 256, 0, s>>>(bg, gout_cs, gout_off, cout,
                                                                                   np, db);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return PIC_ECUDA;
  int e = 0;
  if (cudaMemcpy(&e, err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return PIC_ECUDA;
  if (e) {
    picgb::note(cudaErrorTimeout, ("tcgen05 weight gradient wait " + std::to_string(e)).c_str());
    return PIC_ETIMEOUT;
  }
  return PIC_OK;
}

pic_status pic_upconv_back_bf16(int32_t impl, int32_t B, int32_t H, int32_t W, const void *gout,
                                int32_t gout_cs, int32_t gout_off, int32_t cout, const float *w, void *gin,
                                int32_t cin, void *stream) {
  if (!gout || !w || !gin || B < 1 || H < 1 || W < 1 || cin < 1 || cout < 1 || gout_off < 0 ||
      gout_off + cout > gout_cs || impl < 0 || impl > 1 || (long long)B * H * W * 4 >= (1LL << 31))
    return PIC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bf16 *bg = static_cast<const bf16 *>(gout);
  bf16 *bin = static_cast<bf16 *>(gin);
  if (impl == 1) {
    k_up_back_data<<<gridn((long long)B * H * W * cin), 256, 0, s>>>(bg, gout_cs, gout_off, cout, w, bin, cin,
                                                                    B, H, W);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return PIC_ECUDA;
    return PIC_OK;
  }
  if (!picgb::conv3x3_tc_supported(cout, cin, gout_cs, gout_off, cin, 0, W)) return PIC_EINVAL;
  int *err = nullptr;
  if (cudaGetSymbolAddress((void **)&err, g_conv_err) != cudaSuccess) return PIC_ECUDA;
  const long long nw = 4LL * cin * cout;
  bf16 *wb = nullptr;
  if (cudaMalloc(&wb, size_t(nw) * 2) != cudaSuccess) return PIC_ENOMEM;
  picgb::ConvTC c;
  c.in = bg;
  c.in_cs = gout_cs;
  c.in_off = gout_off;
  c.cin = cout;
  c.w = wb;
  c.bias = nullptr;
  c.out = bin;
  c.out_cs = cin;
  c.out_off = 0;
  c.cout = cin;
  c.B = B;
  c.H = H;
  c.W = W;
  c.relu = 0;
  c.err = err;
  k_to_bf16<<<gridn(nw), 256, 0, s>>>(w, wb, nw);
  pic_status st = PIC_OK;
  if (cudaGetLastError() != cudaSuccess || cudaMemsetAsync(err, 0, 4, s) != cudaSuccess ||
      picgb::conv_upback_tc(c, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    st = PIC_ECUDA;
  int e = 0;
  if (st == PIC_OK && cudaMemcpy(&e, err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) st = PIC_ECUDA;
  cudaFree(wb);
  if (st == PIC_OK && e) {
    picgb::note(cudaErrorTimeout, ("tcgen05 convolution wait " + std::to_string(e)).c_str());
    st = PIC_ETIMEOUT;
  }
  return st;
}

pic_status pic_unet_set_conv_impl(pic_unet *u, int32_t impl) {
  if (!u || impl < 0 || impl > 1) return PIC_EINVAL;
  if (cudaStreamSynchronize(u->stream) != cudaSuccess) return PIC_ECUDA;
  u->conv_impl = impl;
  return PIC_OK;
}

pic_status pic_unet_status(pic_unet *u) {
  if (!u) return PIC_EINVAL;
  int err = 0;
  if (cudaStreamSynchronize(u->stream) != cudaSuccess ||
      cudaMemcpy(&err, u->d_err, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return PIC_ECUDA;
  if (err) {
    cudaMemset(u->d_err, 0, 4);
    return PIC_ETIMEOUT;
  }
  return PIC_OK;
}

pic_status pic_unet_free(pic_unet *u) {
  if (!u) return PIC_OK;
  if (u->stream) cudaStreamSynchronize(u->stream);
  for (void *p : u->allocs) cudaFree(p);
  delete u;
  return PIC_OK;
}

}  // extern "C"

namespace picgb {

// y = U(x) queued on the net's stream; the output stays in the net's buffer.
void unet_forward_only(pic_unet *u, const float *x) { unet::forward(u, x, false); }
const float *unet_output(const pic_unet *u) { return u->y; }
int unet_height(const pic_unet *u) { return u->H; }
int unet_width(const pic_unet *u) { return u->W; }
int unet_batch(const pic_unet *u) { return u->B; }
// kernels one forward launches: the input conversion, 14 convolutions, 3
// pools, 3 transposed convolutions and the head
int unet_forward_kernels() { return 1 + 14 + 3 + 3 + 1; }
// copies the FP32 parameters of src into dst (same architecture) on dst's stream
pic_status unet_copy_params(pic_unet *dst, const pic_unet *src) {
  if (dst->nparam != src->nparam) return PIC_EINVAL;
  if (cudaMemcpyAsync(dst->P, src->P, size_t(src->nparam) * 4, cudaMemcpyDeviceToDevice, dst->stream) !=
      cudaSuccess)
    return PIC_ECUDA;
  unet::weights_to_bf16(dst);
  return cudaStreamSynchronize(dst->stream) == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

}  // namespace picgb
