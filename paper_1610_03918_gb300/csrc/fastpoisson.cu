// Direct inner solve of the Poisson correction equation A e = r, A = -Delta_h
// on the free nodes (Eq. 5 with the Dirichlet values lifted into r), for the
// boxes of Sec. III-B and III-C when y is periodic with a power-of-two ny and
// x is bounded: the free nodes are the full rows 1..m (the plasma slab) and,
// with a trench, the interface row xs = m + 1 and the slot rows below it,
// all on the trench's columns [c0, c0 + wc).
//
// Block elimination of the coupled system (unknowns: slab R, interface G,
// slot S; A_RG, A_GS are the -1 couplings across rows m | xs | xs + 1):
//   v_R = A_RR^-1 r_R,   v_S = A_SS^-1 r_S
//   (A_GG - G_R - G_S) u_G = r_G + v_R(row m) + v_S(row xs + 1)
//   u_R = v_R + A_RR^-1 (u_G on row m),   u_S = v_S + A_SS^-1 (u_G on row xs + 1)
// where G_R, G_S are the slab's and the slot's Green's functions on the
// interface columns (precomputed in FP64, the wc x wc Schur complement
// inverted on the host).
//   Slab: a real FFT along y turns A_RR into one tridiagonal system per mode
//     k = 0..ny/2, tridiag(-1, 4 - 2 cos(2 pi k / ny), -1) along x with
//     Dirichlet rows 0 and m + 1, each solved by parallel cyclic reduction in
//     shared memory; the interface term on row m is added in Fourier space
//     through the precomputed column m of each inverse.
//   Slot: a sine transform across its wc columns (Dirichlet walls) gives wc
//     tridiagonal systems along x (Dirichlet bottom row; the interface is a
//     separate unknown), solved together by the same reduction.
// Arithmetic is FP32; the iterative refinement around it (the residual check
// of the solver) certifies the result.  Each kernel adds the correction it
// forms straight into the double-float potential on the nodes it owns (the
// interface row, the slab rows, the slot rows), so the solve needs no
// separate correction pass.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace picgb {
namespace {

constexpr int kFftThreads = 256;
constexpr int kMaxNy = 2048;
constexpr int kMaxRows = 4096;         // rectangle rows (one mode's reduction fits in shared memory)
constexpr int kPcrThreads = 512;
constexpr int kSlotThreads = 256;
constexpr size_t kSmemMax = 200 * 1024;
constexpr int kRound = 2;              // global loads a thread issues before using them

struct FPArgs {
  int ny, nk, logny, m, xs, slot, c0, wc, ms;
  const float2 *tw;
  const float *dk, *z;               // diagonal per slab mode, interface responses
  float2 *vhat;
  const float *phi, *sb, *zs, *sinv; // slot basis, diagonal per sine mode, responses
  const float2 *twc;                 // [wc][nk]: w_k exp(+2 pi i k (c0 + c) / ny) / ny
  float *vs;                         // [wc][ms] solved slot spectra
  float *ug;                         // [wc] interface values
  float2 *fh;                        // [nk] spectrum of the interface values on row m + 1
  float *sh;                         // [wc] sine spectrum of the interface values
  const float *r;
  float2 *pot;                       // the potential (double-float): the correction is added to it
  PoissonState *ps;
};

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 conj2(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float fma_t(float w, float a, float b) { return fmaf(w, a, b); }
__device__ __forceinline__ float2 fma_t(float w, float2 a, float2 b) {
  return make_float2(fmaf(w, a.x, b.x), fmaf(w, a.y, b.y));
}

// Radix-2 Stockham autosort FFT of n = 2^logn complex points in shared memory
// (x holds the input, y is scratch); returns the buffer holding the result.
// Stage with sub-transform length len and stride s = n / len: for p < len/2,
// q < s, with a = x[q + s p], b = x[q + s (p + len/2)]:
//   y[q + s 2p] = a + b,   y[q + s (2p + 1)] = (a - b) w^p,  w = exp(-+2 pi i / len)
// (tw[t] = exp(-2 pi i t / n), so w^p = tw[p s]; conjugated for the inverse).
// Unscaled.
__device__ float2 *fft_smem(float2 *x, float2 *y, const float2 *tw, int n, int logn, bool inverse) {
  for (int ls = 0; ls < logn; ++ls) {
    const int s = 1 << ls, half = n >> (ls + 1);
    for (int t = threadIdx.x; t < (n >> 1); t += blockDim.x) {
      const int p = t >> ls, q = t & (s - 1);
      float2 wp = tw[p * s];
      if (inverse) wp = conj2(wp);
      const float2 a = x[q + s * p], b = x[q + s * (p + half)];
      y[q + s * (2 * p)] = cadd(a, b);
      y[q + s * (2 * p + 1)] = cmul(csub(a, b), wp);
    }
    __syncthreads();
    float2 *tmp = x;
    x = y;
    y = tmp;
  }
  return x;
}

// Rows of a tridiagonal system a_i x_{i-1} + b_i x_i + c_i x_{i+1} = r_i in
// shared memory.
template <typename T>
struct Rows {
  float *a, *b, *c;
  T *r;
};

// Parallel cyclic reduction (Hockney): step s eliminates every row's
// neighbours at distance s = 1, 2, 4, ... from it, with
//   alpha = -a_i / b_{i-s},  gamma = -c_i / b_{i+s},
//   a_i <- alpha a_{i-s},  c_i <- gamma c_{i+s},
//   b_i <- b_i + alpha c_{i-s} + gamma a_{i+s},  r_i <- r_i + alpha r_{i-s} + gamma r_{i+s},
// until no row is coupled; then x_i = r_i / b_i (the quotients use the fast
// reciprocal, about 2 ulp; the refinement around the solve absorbs it).  A
// zero coupling stays zero,
// so independent systems laid end to end (zero a at each first row, zero c at
// each last row) are solved together.  p holds the input, q is scratch; the
// returned pair holds the reduced rows.
template <typename T>
__device__ Rows<T> pcr(Rows<T> p, Rows<T> q, int n) {
  for (int s = 1; s < n; s <<= 1) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const float ai = p.a[i], ci = p.c[i];
      float bi = p.b[i], an = 0.f, cn = 0.f;
      T ri = p.r[i];
      if (ai != 0.f) {
        const float al = __fdividef(-ai, p.b[i - s]);
        an = al * p.a[i - s];
        bi = fmaf(al, p.c[i - s], bi);
        ri = fma_t(al, p.r[i - s], ri);
      }
      if (ci != 0.f) {
        const float ga = __fdividef(-ci, p.b[i + s]);
        cn = ga * p.c[i + s];
        bi = fmaf(ga, p.a[i + s], bi);
        ri = fma_t(ga, p.r[i + s], ri);
      }
      q.a[i] = an;
      q.b[i] = bi;
      q.c[i] = cn;
      q.r[i] = ri;
    }
    __syncthreads();
    const Rows<T> t = p;
    p = q;
    q = t;
  }
  return p;
}

template <typename T>
__device__ Rows<T> carve_rows(float *&base, int n) {
  Rows<T> r;
  r.a = base;
  r.b = base + n;
  r.c = base + 2 * n;
  r.r = reinterpret_cast<T *>(base + 3 * n + (n & 1) * (sizeof(T) == 8 ? 1 : 0));
  base = reinterpret_cast<float *>(r.r + n);
  return r;
}

// Forward transforms of rectangle rows i0 = 2b + 1 and i1 = i0 + 1, packed as
// one complex sequence z = r_i0 + i r_i1 and separated by the symmetry of real
// transforms: X_a[k] = (Z[k] + conj Z[-k]) / 2, X_b[k] = (Z[k] - conj Z[-k]) / 2i.
__global__ void __launch_bounds__(kFftThreads) k_fp_forward(FPArgs f) {
  extern __shared__ float2 sm[];
  float2 *x = sm, *y = sm + f.ny, *tw = sm + 2 * f.ny;
  for (int t = threadIdx.x; t < (f.ny >> 1); t += blockDim.x) tw[t] = f.tw[t];
  pdl_enter();
  const int i0 = 2 * blockIdx.x + 1, i1 = i0 + 1;
  const bool two = i1 <= f.m;
  constexpr int R = 8;
  for (int j0 = threadIdx.x; j0 < f.ny; j0 += R * blockDim.x) {   // a round's loads in flight together
    float2 v[R];
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const int j = j0 + u * blockDim.x;
      v[u] = j < f.ny ? make_float2(f.r[i0 * f.ny + j], two ? f.r[i1 * f.ny + j] : 0.f) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < R; ++u)
      if (j0 + u * int(blockDim.x) < f.ny) x[j0 + u * blockDim.x] = v[u];
  }
  __syncthreads();
  const float2 *Z = fft_smem(x, y, tw, f.ny, f.logny, false);
  for (int k = threadIdx.x; k < f.nk; k += blockDim.x) {
    const float2 zk = Z[k], zc = conj2(Z[(f.ny - k) & (f.ny - 1)]);
    const float2 d = csub(zk, zc);
    f.vhat[(i0 - 1) * f.nk + k] = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y + zc.y));
    if (two) f.vhat[(i1 - 1) * f.nk + k] = make_float2(0.5f * d.y, -0.5f * d.x);
  }
}

// One tridiagonal system per CTA by parallel cyclic reduction.  CTAs 0..nk-1
// take the slab modes: tridiag(-1, d_k, -1) along x (rows 1..m, Dirichlet rows
// 0 and m + 1), in place on column k of vhat.  CTAs nk..nk+wc-1 take the slot's
// sine modes p: the spectrum sum_c r(xs + 1 + i, c0 + c) phi[p][c] of its rows,
// then tridiag(-1, sb_p, -1) along them, into vs[p].  The matrices do not
// change during a solve, so they are laid out before the wait for the
// preceding kernel.
__global__ void __launch_bounds__(kPcrThreads) k_fp_tridiag(FPArgs f) {
  extern __shared__ float smt[];
  const bool slab = int(blockIdx.x) < f.nk;
  const int n = slab ? f.m : f.ms, k = blockIdx.x, pm = blockIdx.x - f.nk;
  float *base = smt;
  if (slab) {
    const Rows<float2> p = carve_rows<float2>(base, n), q = carve_rows<float2>(base, n);
    const float d = __ldg(f.dk + k);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      p.a[i] = i > 0 ? -1.f : 0.f;
      p.b[i] = d;
      p.c[i] = i + 1 < n ? -1.f : 0.f;
    }
    pdl_enter();
    for (int i0 = threadIdx.x; i0 < n; i0 += kRound * blockDim.x) {
      float2 v[kRound];
#pragma unroll
      for (int u = 0; u < kRound; ++u) {
        const int i = i0 + u * blockDim.x;
        v[u] = i < n ? f.vhat[i * f.nk + k] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < kRound; ++u)
        if (i0 + u * int(blockDim.x) < n) p.r[i0 + u * blockDim.x] = v[u];
    }
    __syncthreads();
    const Rows<float2> x = pcr(p, q, n);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const float2 r = x.r[i];
      const float rb = 1.f / x.b[i];
      f.vhat[i * f.nk + k] = make_float2(r.x * rb, r.y * rb);
    }
  } else {
    const Rows<float> p = carve_rows<float>(base, n), q = carve_rows<float>(base, n);
    float *ph = base;                // [wc] row pm of the sine basis
    const float d = __ldg(f.sb + pm);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      p.a[i] = i > 0 ? -1.f : 0.f;
      p.b[i] = d;
      p.c[i] = i + 1 < n ? -1.f : 0.f;
    }
    for (int c = threadIdx.x; c < f.wc; c += blockDim.x) ph[c] = __ldg(f.phi + pm * f.wc + c);
    pdl_enter();
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const float *rr = f.r + (f.xs + 1 + i) * f.ny + f.c0;
      float acc = 0.f;
      for (int c0 = 0; c0 < f.wc; c0 += kRound) {
        float v[kRound];
#pragma unroll
        for (int u = 0; u < kRound; ++u) v[u] = c0 + u < f.wc ? __ldg(rr + c0 + u) : 0.f;
#pragma unroll
        for (int u = 0; u < kRound; ++u)
          if (c0 + u < f.wc) acc = fmaf(v[u], ph[c0 + u], acc);
      }
      p.r[i] = acc;
    }
    __syncthreads();
    const Rows<float> x = pcr(p, q, n);
    for (int i = threadIdx.x; i < n; i += blockDim.x) f.vs[pm * n + i] = x.r[i] / x.b[i];
  }
}

// Interface, one CTA: g = r_G + v_R(row m) + v_S(first slot row) on the
// interface columns (v_R by the inverse DFT of the solved spectra of row m,
// v_S from the solved slot spectra), then u_G = S^-1 g, written to ug and to
// e on the interface.  The corrections that u_G makes to the slab and the
// slot are applied by the inverse-transform kernel.  The sine basis and
// S^-1 are staged before the wait for the solves; a warp per column forms
// its sums across its lanes.
__global__ void __launch_bounds__(kSlotThreads) k_fp_interface(FPArgs f) {
  extern __shared__ float ss[];
  const int wc = f.wc, ms = f.ms, ny = f.ny, nk = f.nk;
  float *sphi = ss;                  // [wc][wc] sine basis
  float *sinv = sphi + wc * wc;      // [wc][wc] S^-1
  float *gv = sinv + wc * wc;        // [wc] interface right-hand side g
  for (int t = threadIdx.x; t < wc * wc; t += blockDim.x) {
    sphi[t] = __ldg(f.phi + t);
    sinv[t] = __ldg(f.sinv + t);
  }
  if (threadIdx.x == 0) {   // the DFT weights into L2 while the solves finish
    const unsigned bytes = unsigned(size_t(wc) * nk * sizeof(float2)) & ~15u;
    if (bytes) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(f.twc), "r"(bytes) : "memory");
  }
  pdl_enter();
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const float2 *vm = f.vhat + size_t(f.m - 1) * nk;
  constexpr int U = 8;   // loads of a round in flight together
  for (int c = warp; c < wc; c += nw) {
    const float2 *tc = f.twc + size_t(c) * nk;
    float acc = 0.f;
    for (int k0 = lane; k0 < nk; k0 += 32 * U) {
      float2 v[U], t[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int k = k0 + 32 * u;
        v[u] = k < nk ? vm[k] : make_float2(0.f, 0.f);
        t[u] = k < nk ? __ldg(tc + k) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) acc = fmaf(v[u].x, t[u].x, fmaf(-v[u].y, t[u].y, acc));
    }
    for (int pm = lane; pm < wc; pm += 32) acc = fmaf(f.vs[pm * ms], sphi[pm * wc + c], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) gv[c] = f.r[f.xs * ny + f.c0 + c] + acc;
  }
  __syncthreads();
  float *ugs = gv + wc;              // [wc] u_G
  for (int c = threadIdx.x; c < wc; c += blockDim.x) {
    float acc = 0.f;
    for (int qq = 0; qq < wc; ++qq) acc = fmaf(sinv[c * wc + qq], gv[qq], acc);
    ugs[c] = acc;
    f.ug[c] = acc;
    const int n = f.xs * ny + f.c0 + c;
    f.pot[n] = pair_add_f(f.pot[n], acc);
  }
  __syncthreads();
  // the spectra of u_G the inverse-transform kernel applies: fh[k] = sum_c
  // u_G(c) exp(-2 pi i k (c0 + c) / ny) and sh[p] = sum_c phi[p][c] u_G(c)
  // (from the weights above: exp(-2 pi i k j / ny) = conj(twc[c][k]) ny / w_k)
  for (int k = threadIdx.x; k < nk; k += blockDim.x) {
    float2 h = make_float2(0.f, 0.f);
    for (int c0 = 0; c0 < wc; c0 += U) {
      float2 w[U];
#pragma unroll
      for (int u = 0; u < U; ++u) w[u] = c0 + u < wc ? __ldg(f.twc + size_t(c0 + u) * nk + k) : make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const float g = c0 + u < wc ? ugs[c0 + u] : 0.f;
        h.x = fmaf(g, w[u].x, h.x);
        h.y = fmaf(-g, w[u].y, h.y);
      }
    }
    const float sc = float(ny) / ((k == 0 || k == nk - 1) ? 1.f : 2.f);
    f.fh[k] = make_float2(h.x * sc, h.y * sc);
  }
  for (int pm = threadIdx.x; pm < wc; pm += blockDim.x) {
    float acc = 0.f;
    for (int c = 0; c < wc; ++c) acc = fmaf(sphi[pm * wc + c], ugs[c], acc);
    f.sh[pm] = acc;
  }
  if (threadIdx.x == 0) {
    f.ps->inner_iters += 1;
    f.ps->total_iters += 1;
  }
}

// Inverse transforms of rows i0, i1 (with the interface term z_k(i) fhat[k]
// when there is a slot, fhat[k] = sum_c u_G(c) exp(-2 pi i k (c0 + c) / ny)
// formed here from u_G): Z[k] = X_a[k] + i X_b[k] over the full spectrum
// (X[-k] = conj X[k]), e(i0) = Re IFFT(Z) / ny, e(i1) = Im IFFT(Z) / ny.
// The CTAs after the slab's take the slot rows: with the sine spectrum
// sh[p] = sum_c phi[p][c] u_G(c), e(row, c) = sum_p (v_S[p][row] +
// zs[p][row] sh[p]) phi[p][c].
__global__ void __launch_bounds__(kFftThreads) k_fp_inverse(FPArgs f) {
  extern __shared__ float2 sm[];
  const int rows = (f.m + 1) / 2, wc = f.wc;
  if (int(blockIdx.x) >= rows) {
    float *sphi = reinterpret_cast<float *>(sm), *sh = sphi + wc * wc;
    for (int t = threadIdx.x; t < wc * wc; t += blockDim.x) sphi[t] = __ldg(f.phi + t);
    pdl_enter();
    for (int pm = threadIdx.x; pm < wc; pm += blockDim.x) sh[pm] = f.sh[pm];
    __syncthreads();
    const int t = (blockIdx.x - rows) * blockDim.x + threadIdx.x;
    if (t < f.ms * wc) {
      const int row = t / wc, c = t - row * wc;
      float acc = 0.f;
      for (int p0 = 0; p0 < wc; p0 += kRound) {   // a round's loads in flight together
        float zv[kRound], vv[kRound];
#pragma unroll
        for (int u = 0; u < kRound; ++u) {
          const int pm = p0 + u;
          zv[u] = pm < wc ? __ldg(f.zs + pm * f.ms + row) : 0.f;
          vv[u] = pm < wc ? f.vs[pm * f.ms + row] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kRound; ++u)
          if (p0 + u < wc) acc = fmaf(fmaf(zv[u], sh[p0 + u], vv[u]), sphi[(p0 + u) * wc + c], acc);
      }
      const int n = (f.xs + 1 + row) * f.ny + f.c0 + c;
      f.pot[n] = pair_add_f(f.pot[n], acc);
    }
    return;
  }
  float2 *x = sm, *y = sm + f.ny, *tw = sm + 2 * f.ny;
  for (int t = threadIdx.x; t < (f.ny >> 1); t += blockDim.x) tw[t] = f.tw[t];
  const int i0 = 2 * blockIdx.x + 1, i1 = i0 + 1;
  const bool two = i1 <= f.m;
  if (f.slot && threadIdx.x == 0) {
    // this row pair's interface responses (a static table) into L2 meanwhile:
    // the 16-byte aligned part of z[i0 - 1 .. i1 - 1][*]
    const uintptr_t lo = (reinterpret_cast<uintptr_t>(f.z + size_t(i0 - 1) * f.nk) + 15) & ~uintptr_t(15);
    const uintptr_t hi = reinterpret_cast<uintptr_t>(f.z + size_t(two ? i1 : i0) * f.nk) & ~uintptr_t(15);
    if (hi > lo)
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"(unsigned(hi - lo)) : "memory");
  }
  pdl_enter();
  // the potential of this thread's output nodes, read early (its loads
  // overlap the spectra's); the row pair has at most kMaxNy / blockDim.x
  // nodes per thread and row
  constexpr int kOut = kMaxNy / kFftThreads;
  float2 p0[kOut], p1[kOut];
#pragma unroll
  for (int u = 0; u < kOut; ++u) {
    const int j = threadIdx.x + u * kFftThreads;
    p0[u] = j < f.ny ? f.pot[i0 * f.ny + j] : make_float2(0.f, 0.f);
    p1[u] = j < f.ny && two ? f.pot[i1 * f.ny + j] : make_float2(0.f, 0.f);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // this pass's correction is in the potential once this kernel is done
    f.ps->outer_iters += 1;
    if (!f.slot) {
      f.ps->inner_iters += 1;
      f.ps->total_iters += 1;
    }
  }
  for (int k0 = threadIdx.x; k0 < f.nk; k0 += kRound * blockDim.x) {
    float2 av[kRound], bv[kRound], hv[kRound];
    float za[kRound], zb[kRound];
#pragma unroll
    for (int u = 0; u < kRound; ++u) {   // a round's loads in flight together
      const int k = k0 + u * blockDim.x;
      const bool in = k < f.nk;
      av[u] = in ? f.vhat[(i0 - 1) * f.nk + k] : make_float2(0.f, 0.f);
      bv[u] = in && two ? f.vhat[(i1 - 1) * f.nk + k] : make_float2(0.f, 0.f);
      hv[u] = in && f.slot ? f.fh[k] : make_float2(0.f, 0.f);
      za[u] = in && f.slot ? __ldg(f.z + (i0 - 1) * f.nk + k) : 0.f;
      zb[u] = in && f.slot && two ? __ldg(f.z + (i1 - 1) * f.nk + k) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kRound; ++u) {
      const int k = k0 + u * blockDim.x;
      if (k >= f.nk) continue;
      // the interface term z_k(i) fhat[k] (zero without a slot)
      const float2 a = make_float2(fmaf(za[u], hv[u].x, av[u].x), fmaf(za[u], hv[u].y, av[u].y));
      const float2 b = make_float2(fmaf(zb[u], hv[u].x, bv[u].x), fmaf(zb[u], hv[u].y, bv[u].y));
      // Z[k] = a + i b, Z[ny - k] = conj(a) + i conj(b)
      x[k] = make_float2(a.x - b.y, a.y + b.x);
      if (k > 0 && k < f.ny - k) x[f.ny - k] = make_float2(a.x + b.y, -a.y + b.x);
    }
  }
  __syncthreads();
  const float2 *Z = fft_smem(x, y, tw, f.ny, f.logny, true);
  const float s = 1.f / float(f.ny);
#pragma unroll
  for (int u = 0; u < kOut; ++u) {
    const int j = threadIdx.x + u * kFftThreads;
    if (j < f.ny) {
      f.pot[i0 * f.ny + j] = pair_add_f(p0[u], Z[j].x * s);
      if (two) f.pot[i1 * f.ny + j] = pair_add_f(p1[u], Z[j].y * s);
    }
  }
}

FPArgs fp_args(pic_ctx *c, const float *r, float2 *pot, PoissonState *ps) {
  const FastPoisson &p = c->fp;
  FPArgs a;
  a.ny = p.ny;
  a.nk = p.nk;
  a.logny = p.logny;
  a.m = p.m;
  a.xs = p.xs;
  a.slot = p.slot;
  a.c0 = p.c0;
  a.wc = p.wc;
  a.ms = p.ms;
  a.tw = p.tw;
  a.dk = p.dk;
  a.z = p.z;
  a.vhat = p.vhat;
  a.phi = p.phi;
  a.vs = p.vs;
  a.ug = p.ug;
  a.sb = p.sb;
  a.zs = p.zs;
  a.sinv = p.sinv;
  a.twc = p.twc;
  a.fh = p.fh;
  a.sh = p.sh;
  a.r = r;
  a.pot = pot;
  a.ps = ps;
  return a;
}

size_t fft_smem_bytes(int ny, int wc) {
  return std::max(size_t(2 * ny + ny / 2) * sizeof(float2) + size_t(wc) * 4,
                  (size_t(wc) * wc + 2 * size_t(wc)) * 4);
}
// two Rows<T> sets of n rows (with the alignment padding of carve_rows)
size_t rows_bytes(int n, size_t tsize) { return 2 * (size_t(3 * n + (n & 1)) * 4 + size_t(n) * tsize); }
size_t tridiag_smem_bytes(int m, int ms, int wc) {
  return std::max(rows_bytes(m, sizeof(float2)), rows_bytes(ms, 4) + size_t(wc) * 4);
}
size_t slot_smem_bytes(int wc) { return (2 * size_t(wc) * wc + 2 * size_t(wc)) * 4; }

// Thomas factors of tridiag(-1, d, -1) of size n: w_1 = 1/d, w_i = 1/(d - w_{i-1})
void thomas_factors(double d, int n, double *w) {
  double v = 1.0 / d;
  w[0] = v;
  for (int i = 1; i < n; ++i) {
    v = 1.0 / (d - v);
    w[i] = v;
  }
}

// Solution of tridiag(-1, d, -1) x = rhs with the factors above (FP64)
void thomas_solve(const double *w, int n, const double *rhs, double *x) {
  std::vector<double> y(n);
  double prev = 0.0;
  for (int i = 0; i < n; ++i) {
    prev = w[i] * (rhs[i] + prev);
    y[i] = prev;
  }
  double nxt = 0.0;
  for (int i = n - 1; i >= 0; --i) {
    nxt = y[i] + w[i] * nxt;
    x[i] = nxt;
  }
}

bool invert(std::vector<double> &A, int n, std::vector<double> &inv) {
  inv.assign(size_t(n) * n, 0.0);
  for (int r = 0; r < n; ++r) inv[size_t(r) * n + r] = 1.0;
  for (int col = 0; col < n; ++col) {   // Gauss-Jordan with partial pivoting
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(A[size_t(r) * n + col]) > std::fabs(A[size_t(piv) * n + col])) piv = r;
    if (!(std::fabs(A[size_t(piv) * n + col]) > 1e-300)) return false;
    if (piv != col)
      for (int k = 0; k < n; ++k) {
        std::swap(A[size_t(piv) * n + k], A[size_t(col) * n + k]);
        std::swap(inv[size_t(piv) * n + k], inv[size_t(col) * n + k]);
      }
    const double d = A[size_t(col) * n + col];
    for (int k = 0; k < n; ++k) {
      A[size_t(col) * n + k] /= d;
      inv[size_t(col) * n + k] /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double q = A[size_t(r) * n + col];
      if (q == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        A[size_t(r) * n + k] -= q * A[size_t(col) * n + k];
        inv[size_t(r) * n + k] -= q * inv[size_t(col) * n + k];
      }
    }
  }
  return true;
}

template <typename T>
T *upload(pic_ctx *c, const std::vector<T> &v) {
  T *d = static_cast<T *>(dev_alloc(c, std::max<size_t>(v.size(), 1) * sizeof(T)));
  if (d && !v.empty()) cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  return d;
}

}  // namespace

cudaError_t fast_poisson_setup(pic_ctx *c) {
  FastPoisson &p = c->fp;
  p = FastPoisson();
  const Geom &g = c->g;
  if (c->cfg.poisson_method != 0 || g.px || !g.py) return cudaSuccess;
  const int ny = g.nyn, nxn = g.nxn;
  if (ny < 4 || ny > kMaxNy || (ny & (ny - 1))) return cudaSuccess;
  auto free_at = [&](int i, int j) { return (c->h_nodeflags[size_t(i) * ny + j] & kFree) != 0; };
  auto row_count = [&](int i) {
    int n = 0;
    for (int j = 0; j < ny; ++j) n += free_at(i, j);
    return n;
  };
  if (row_count(0) != 0 || row_count(nxn - 1) != 0) return cudaSuccess;
  int xs = 1;
  while (xs < nxn - 1 && row_count(xs) == ny) ++xs;
  const int m = xs - 1;
  if (m < 1 || m > kMaxRows || tridiag_smem_bytes(m, 0, 0) > kSmemMax) return cudaSuccess;
  int c0 = 0, wc = 0, ms = 0;
  // a slot exists when some row from xs on still has free nodes (a trench
  // one cell wide has none: its walls' nodes are all on the conductor)
  bool slot = false;
  for (int r = xs; r < nxn; ++r) slot = slot || row_count(r) > 0;
  if (slot) {
    // the interface row's free nodes: one run of columns with a wall on each side
    int first = -1, last = -1;
    for (int j = 0; j < ny; ++j)
      if (free_at(xs, j)) {
        if (first < 0) first = j;
        last = j;
      }
    if (first < 1 || last > ny - 2) return cudaSuccess;
    c0 = first;
    wc = last - first + 1;
    if (row_count(xs) != wc) return cudaSuccess;
    // slot rows: the same columns, down to the last free row
    int r = xs + 1;
    while (r < nxn - 1 && row_count(r) > 0) {
      if (row_count(r) != wc) return cudaSuccess;
      for (int j = c0; j < c0 + wc; ++j)
        if (!free_at(r, j)) return cudaSuccess;
      ++r;
    }
    for (int rr = r; rr < nxn; ++rr)
      if (row_count(rr) != 0) return cudaSuccess;
    ms = r - xs - 1;
    if (ms < 1 || tridiag_smem_bytes(0, ms, wc) > kSmemMax || slot_smem_bytes(wc) > kSmemMax)
      return cudaSuccess;
  }
  const int nk = ny / 2 + 1;
  int logny = 0;
  while ((1 << logny) < ny) ++logny;
  const double pi = 3.14159265358979323846;
  // twiddles, the slab modes' diagonals and (with a slot) the column m of
  // each mode's inverse, by the Thomas recursion in FP64
  std::vector<float2> tw(ny);
  for (int t = 0; t < ny; ++t)
    tw[t] = make_float2(float(std::cos(2 * pi * t / ny)), float(-std::sin(2 * pi * t / ny)));
  std::vector<double> wk(m), col(m), rhs(m, 0.0);
  std::vector<float> dk(nk), z;
  std::vector<double> zlast(nk);   // [T_k^-1]_{m,m}
  if (slot) z.resize(size_t(m) * nk);
  rhs[m - 1] = 1.0;
  for (int k = 0; k < nk; ++k) {
    const double d = 4.0 - 2.0 * std::cos(2 * pi * k / ny);
    dk[k] = float(d);
    if (slot) {
      thomas_factors(d, m, wk.data());
      thomas_solve(wk.data(), m, rhs.data(), col.data());
      for (int i = 0; i < m; ++i) z[size_t(i) * nk + k] = float(col[i]);
      zlast[k] = col[m - 1];
    }
  }
  p.tw = upload(c, tw);
  p.dk = upload(c, dk);
  p.vhat = static_cast<float2 *>(dev_alloc(c, size_t(m) * nk * sizeof(float2)));
  if (!p.tw || !p.dk || !p.vhat) return cudaErrorMemoryAllocation;
  if (slot) {
    // slot: orthonormal sine basis across the columns, the diagonal of each
    // sine mode's system along its rows and the responses to a unit value on
    // its first row ([mode][row])
    std::vector<double> phi(size_t(wc) * wc), mu(wc);
    for (int q = 0; q < wc; ++q) {
      mu[q] = 2.0 - 2.0 * std::cos(pi * (q + 1) / (wc + 1));
      for (int cc = 0; cc < wc; ++cc)
        phi[size_t(q) * wc + cc] = std::sqrt(2.0 / (wc + 1)) * std::sin(pi * (q + 1) * (cc + 1) / (wc + 1));
    }
    std::vector<float> sbf(wc), zsf(size_t(ms) * wc), phif(phi.begin(), phi.end());
    std::vector<double> wsk(ms), zcol(ms), e0(ms, 0.0), zfirst(wc);
    e0[0] = 1.0;
    for (int q = 0; q < wc; ++q) {
      sbf[q] = float(2.0 + mu[q]);
      thomas_factors(2.0 + mu[q], ms, wsk.data());
      thomas_solve(wsk.data(), ms, e0.data(), zcol.data());
      for (int i = 0; i < ms; ++i) zsf[size_t(q) * ms + i] = float(zcol[i]);
      zfirst[q] = zcol[0];
    }
    // Schur complement on the interface: A_GG - G_R - G_S
    std::vector<double> S(size_t(wc) * wc, 0.0), Sinv;
    for (int a = 0; a < wc; ++a) {
      S[size_t(a) * wc + a] = 4.0;
      if (a > 0) S[size_t(a) * wc + a - 1] = -1.0;
      if (a + 1 < wc) S[size_t(a) * wc + a + 1] = -1.0;
      for (int b = 0; b < wc; ++b) {
        double gr = 0.0;
        for (int k = 0; k < nk; ++k) {
          const double wgt = (k == 0 || k == nk - 1) ? 1.0 : 2.0;
          gr += wgt * zlast[k] * std::cos(2 * pi * double(k) * double(a - b) / ny);
        }
        gr /= ny;
        double gs = 0.0;
        for (int q = 0; q < wc; ++q) gs += phi[size_t(q) * wc + a] * zfirst[q] * phi[size_t(q) * wc + b];
        S[size_t(a) * wc + b] -= gr + gs;
      }
    }
    if (!invert(S, wc, Sinv)) return cudaSuccess;   // cannot happen for an SPD system; keep the V-cycle
    std::vector<float> sinvf(Sinv.begin(), Sinv.end());
    // inverse-DFT weights of the interface columns: w_k = 1 for k = 0 and
    // k = ny / 2, 2 between (a real row's spectrum holds k <= ny / 2)
    std::vector<float2> twc(size_t(wc) * nk);
    for (int cc = 0; cc < wc; ++cc)
      for (int k = 0; k < nk; ++k) {
        const double wgt = (k == 0 || k == nk - 1) ? 1.0 : 2.0;
        const double ang = 2 * pi * double((int64_t(k) * (c0 + cc)) % ny) / ny;
        twc[size_t(cc) * nk + k] = make_float2(float(wgt * std::cos(ang) / ny), float(wgt * std::sin(ang) / ny));
      }
    p.z = upload(c, z);
    p.phi = upload(c, phif);
    p.sb = upload(c, sbf);
    p.zs = upload(c, zsf);
    p.sinv = upload(c, sinvf);
    p.twc = upload(c, twc);
    p.vs = static_cast<float *>(dev_alloc(c, size_t(wc) * ms * sizeof(float)));
    p.ug = static_cast<float *>(dev_alloc(c, size_t(wc) * sizeof(float)));
    p.fh = static_cast<float2 *>(dev_alloc(c, size_t(nk) * sizeof(float2)));
    p.sh = static_cast<float *>(dev_alloc(c, size_t(wc) * sizeof(float)));
    if (!p.z || !p.phi || !p.sb || !p.zs || !p.sinv || !p.twc || !p.vs || !p.ug || !p.fh || !p.sh)
      return cudaErrorMemoryAllocation;
  }
  p.ny = ny;
  p.nk = nk;
  p.logny = logny;
  p.m = m;
  p.xs = xs;
  p.slot = slot ? 1 : 0;
  p.c0 = c0;
  p.wc = wc;
  p.ms = ms;
  p.kernels = slot ? 4 : 3;
  // dynamic shared memory beyond the default 48 KB (granted per kernel, so
  // the largest size any context may use)
  cudaError_t e = cudaFuncSetAttribute(k_fp_tridiag, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(kSmemMax));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fp_interface, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSmemMax));
  if (e != cudaSuccess) return e;
  p.enabled = 1;
  return cudaGetLastError();
}

void fast_poisson_launch(pic_ctx *c, const float *r, float2 *pot, PoissonState *ps) {
  const FPArgs a = fp_args(c, r, pot, ps);
  const int rows = (a.m + 1) / 2;
  launch(k_fp_forward, rows, kFftThreads, fft_smem_bytes(a.ny, a.wc), c->stream, a);
  launch(k_fp_tridiag, a.nk + (a.slot ? a.wc : 0), kPcrThreads,
         tridiag_smem_bytes(a.m, a.slot ? a.ms : 0, a.wc), c->stream, a);
  if (a.slot) launch(k_fp_interface, 1, kSlotThreads, slot_smem_bytes(a.wc), c->stream, a);
  const int slot_ctas = a.slot ? (a.ms * a.wc + kFftThreads - 1) / kFftThreads : 0;
  launch(k_fp_inverse, rows + slot_ctas, kFftThreads, fft_smem_bytes(a.ny, a.wc), c->stream, a);
  c->launches += c->fp.kernels;
}

}  // namespace picgb
