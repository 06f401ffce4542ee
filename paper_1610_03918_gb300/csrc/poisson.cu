// Field side of the step: charge density, the Poisson solve of Eq. 5 and
// E = -grad Phi (Sec. II).
//
// rho = sum_s q_s w_s 2^-20 acc_s + rho_ext + bottom surface charge, and on
// the free (non-Dirichlet) nodes b = rho + sum of Dirichlet neighbour values.
// A = -Delta_h (5-point, unit spacing) on the free nodes, periodic where the
// box is.  The solve is an FP64 iterative refinement around an FP32
// multigrid-preconditioned conjugate gradient:
//
//   repeat:  r = b - A phi          (FP64 stencil, FP64 norm: the certificate)
//            stop if ||r|| <= rtol ||b||
//            solve A e = r by PCG   (FP32 vectors and stencils, FP64 dots,
//                                    symmetric geometric V-cycle preconditioner)
//            phi += e                (FP64)
//
// The V-cycle coarsens by 2 with injected Dirichlet masks, rediscretised
// operators (A / h^2), full-weighting restriction, bilinear prolongation
// (restriction = prolongation^T / 4) and red-black Gauss-Seidel smoothing
// (red then black before, black then red after), so the preconditioner is
// symmetric.  Levels with at most kSmallLevel nodes run inside one CTA.
// A doubly periodic box has no Dirichlet node: b loses its mean and the
// preconditioned residual is projected to zero mean.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace picgb {
namespace {

constexpr int kThreads = 256;
constexpr int kSmallLevel = 16384;
constexpr int kCoarseThreads = 1024;
constexpr int kMaxOuter = 8;
constexpr int kCoarsestSweeps = 24;

__device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum of NV doubles over the block; thread 0 gets the result.
template <int NV>
__device__ void block_sum(double (&v)[NV]) {
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k][w] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0;
      for (int q = 0; q < nw; ++q) s += sh[k][q];
      v[k] = s;
    }
  }
  __syncthreads();
}

// Deterministic grid reduction: every block publishes its partials, the
// last block to arrive sums them in block order.  Returns true in the last
// block, where thread 0 holds the totals in v.
template <int NV>
__device__ bool grid_sum(double (&v)[NV], double *part, unsigned int *ticket) {
  __shared__ bool last;
  block_sum<NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) part[blockIdx.x * NV + k] = v[k];
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double s[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) s[k] = 0;
  const volatile double *vp = part;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < NV; ++k) s[k] += vp[b * NV + k];
  }
  block_sum<NV>(s);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = s[k];
    *ticket = 0u;
  }
  return true;
}

struct FineArgs {
  Geom g;
  const uint8_t *flags;
  const double *lift;
  const double *gval;
  double *rho, *b, *phi;
  unsigned long long *acc;
  const double *rho_ext;
  const unsigned long long *bottom;
  double qw[2];              // q_s w_s 2^-20
  double sw[2];              // q_s w_s (surface charge per hit)
  int surface;
  float *r32, *z, *p_old, *p_new, *q, *e;
  double *r64;
  PoissonState *ps;
  double *part;
  unsigned int *ticket;
  int singular;
  double rtol;
  int maxit;
  int32_t *step;
  int advance_step;
  float2 *E;
  double *fe;
};

// acc -> rho, b; clears acc.  For a doubly periodic box the mean of b is kept.
__global__ void k_rho(FineArgs a) {
  const Geom g = a.g;
  const int nn = g.nxn * g.nyn;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  double v[2] = {0.0, 0.0};
  if (n < nn) {
    const unsigned long long a0 = a.acc[n], a1 = a.acc[nn + n];
    a.acc[n] = 0ull;
    a.acc[nn + n] = 0ull;
    double rho = a.rho_ext[n] + a.qw[0] * double(a0) + a.qw[1] * double(a1);
    if (a.surface && !g.px) {
      const int i = n / g.nyn, j = n - (n / g.nyn) * g.nyn;
      if (i == g.nx - 1) {
        // half of bottom face k's charge on nodes (nx-1, k) and (nx-1, k+1)
        double s = 0.0;
        if (j < g.ny) s += 0.5 * (a.sw[0] * double(a.bottom[j]) + a.sw[1] * double(a.bottom[g.ny + j]));
        int jm = j - 1;
        if (g.py && jm < 0) jm += g.ny;
        if (jm >= 0 && jm < g.ny)
          s += 0.5 * (a.sw[0] * double(a.bottom[jm]) + a.sw[1] * double(a.bottom[g.ny + jm]));
        rho += s;
      }
    }
    a.rho[n] = rho;
    const bool fr = a.flags[n] & kFree;
    const double bb = fr ? rho + a.lift[n] : 0.0;
    a.b[n] = bb;
    v[0] = bb;
    v[1] = fr ? 1.0 : 0.0;
  }
  if (grid_sum<2>(v, a.part, a.ticket) && threadIdx.x == 0) {
    a.ps->bmean = a.singular ? v[0] / v[1] : 0.0;
    if (a.advance_step) *a.step += 1;
  }
}

// phi <- Dirichlet values, zero on free nodes (cold start)
__global__ void k_phi_reset(FineArgs a) {
  const int nn = a.g.nxn * a.g.nyn;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < nn) a.phi[n] = a.gval[n];
}

__device__ __forceinline__ void nbr_index(const Geom &g, int n, int &xm, int &xp, int &ym, int &yp) {
  const int i = n / g.nyn, j = n - (n / g.nyn) * g.nyn;
  const int im = g.px ? wrapi(i - 1, g.nxn) : max(i - 1, 0);
  const int ip = g.px ? wrapi(i + 1, g.nxn) : min(i + 1, g.nxn - 1);
  const int jm = g.py ? wrapi(j - 1, g.nyn) : max(j - 1, 0);
  const int jp = g.py ? wrapi(j + 1, g.nyn) : min(j + 1, g.nyn - 1);
  xm = im * g.nyn + j;
  xp = ip * g.nyn + j;
  ym = i * g.nyn + jm;
  yp = i * g.nyn + jp;
}

// Outer FP64 residual r = b - A phi (the certificate) and the set-up of the
// inner PCG on A e = r.
__global__ void k_resid64(FineArgs a) {
  const Geom g = a.g;
  const int nn = g.nxn * g.nyn;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  double v[2] = {0.0, 0.0};
  if (n < nn) {
    float r32 = 0.f;
    if (a.flags[n] & kFree) {
      int xm, xp, ym, yp;
      nbr_index(g, n, xm, xp, ym, yp);
      const double rho = a.b[n] - a.lift[n] - a.ps->bmean;
      const double Aphi = 4.0 * a.phi[n] - a.phi[xm] - a.phi[xp] - a.phi[ym] - a.phi[yp];
      const double r = rho - Aphi;
      r32 = float(r);
      const double bb = a.b[n] - a.ps->bmean;
      v[0] = r * r;
      v[1] = bb * bb;
    }
    a.r32[n] = r32;
    a.e[n] = 0.f;
    a.p_old[n] = 0.f;
  }
  if (grid_sum<2>(v, a.part, a.ticket) && threadIdx.x == 0) {
    PoissonState *ps = a.ps;
    ps->rr64 = v[0];
    ps->bb = v[1];
    ps->rel = v[1] > 0 ? sqrt(v[0] / v[1]) : sqrt(v[0]);
    const bool ok = ps->rel <= a.rtol || v[0] == 0.0;
    ps->outer_done = ok ? 1 : 0;
    ps->inner_done = ok ? 1 : 0;
    ps->inner_iters = 0;
    ps->rr0 = v[0];
    ps->rr = v[0];
    // inner target: bring ||r|| to half the outer target, no tighter than FP32 allows
    double t = 0.5 * a.rtol * sqrt(v[1]) / fmax(sqrt(v[0]), 1e-300);
    ps->tol_in = fmin(fmax(t, 3e-6), 0.5);
    ps->beta = 0.0;
    ps->rz = 0.0;
  }
}

// rz = <r, z - zmean> and zmean (doubly periodic box)
__global__ void k_rz(FineArgs a) {
  if (a.ps->inner_done) return;
  const int nn = a.g.nxn * a.g.nyn;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  double v[3] = {0.0, 0.0, 0.0};
  if (n < nn) {
    const double r = a.r32[n], z = a.z[n];
    v[0] = r * z;
    v[1] = z;
    v[2] = r;
  }
  if (grid_sum<3>(v, a.part, a.ticket) && threadIdx.x == 0) {
    PoissonState *ps = a.ps;
    const double zm = a.singular ? v[1] / double(nn) : 0.0;
    ps->zmean = zm;
    ps->rz_old = ps->rz;
    ps->rz = v[0] - zm * v[2];
  }
}

// p_new = (z - zmean) + beta p_old, q = A p_new, pq = <p_new, q>
__global__ void k_pq(FineArgs a) {
  const PoissonState *ps = a.ps;
  if (ps->inner_done) return;
  const Geom g = a.g;
  const int nn = g.nxn * g.nyn;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const float beta = ps->inner_iters == 0 ? 0.f : float(ps->rz / ps->rz_old);
  const float zm = float(ps->zmean);
  double v[1] = {0.0};
  if (n < nn) {
    float pn = 0.f, qn = 0.f;
    if (a.flags[n] & kFree) {
      int xm, xp, ym, yp;
      nbr_index(g, n, xm, xp, ym, yp);
      auto P = [&](int m) -> float {
        return (a.flags[m] & kFree) ? (a.z[m] - zm) + beta * a.p_old[m] : 0.f;
      };
      pn = P(n);
      qn = 4.f * pn - P(xm) - P(xp) - P(ym) - P(yp);
      v[0] = double(pn) * double(qn);
    }
    a.p_new[n] = pn;
    a.q[n] = qn;
  }
  if (grid_sum<1>(v, a.part, a.ticket) && threadIdx.x == 0) a.ps->pq = v[0];
}

// e += alpha p, r -= alpha q, rr = <r, r>; convergence of the inner solve
__global__ void k_update(FineArgs a) {
  PoissonState *ps = a.ps;
  if (ps->inner_done) return;
  const int nn = a.g.nxn * a.g.nyn;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const float alpha = float(ps->rz / ps->pq);
  double v[1] = {0.0};
  if (n < nn) {
    const float p = a.p_new[n];
    a.e[n] += alpha * p;
    const float r = a.r32[n] - alpha * a.q[n];
    a.r32[n] = r;
    a.p_old[n] = p;
    v[0] = double(r) * double(r);
  }
  if (grid_sum<1>(v, a.part, a.ticket) && threadIdx.x == 0) {
    ps->rr = v[0];
    ps->inner_iters += 1;
    ps->total_iters += 1;
    const double tol = ps->tol_in;
    if (sqrt(v[0]) <= tol * sqrt(ps->rr0) || ps->inner_iters >= a.maxit || !(v[0] == v[0]))
      ps->inner_done = 1;
  }
}

__global__ void k_set_status(uint32_t *st, uint32_t bit) { atomicOr(st, bit); }

__global__ void k_correct(FineArgs a) {
  const int nn = a.g.nxn * a.g.nyn;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < nn && (a.flags[n] & kFree)) a.phi[n] += double(a.e[n]);
}

// E = -grad phi by the open-edge rule; field energy 1/2 sum |E|^2
__global__ void k_field(FineArgs a) {
  const Geom g = a.g;
  const int nn = g.nxn * g.nyn;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  double v[1] = {0.0};
  if (n < nn) {
    const uint8_t f = a.flags[n];
    const int i = n / g.nyn, j = n - (n / g.nyn) * g.nyn;
    const double p = a.phi[n];
    double sx = 0.0, sy = 0.0;
    int cx = 0, cy = 0;
    if (f & kOpenXm) { sx += p - a.phi[(g.px ? wrapi(i - 1, g.nxn) : i - 1) * g.nyn + j]; ++cx; }
    if (f & kOpenXp) { sx += a.phi[(g.px ? wrapi(i + 1, g.nxn) : i + 1) * g.nyn + j] - p; ++cx; }
    if (f & kOpenYm) { sy += p - a.phi[i * g.nyn + (g.py ? wrapi(j - 1, g.nyn) : j - 1)]; ++cy; }
    if (f & kOpenYp) { sy += a.phi[i * g.nyn + (g.py ? wrapi(j + 1, g.nyn) : j + 1)] - p; ++cy; }
    const double ex = cx ? -sx / cx : 0.0;
    const double ey = cy ? -sy / cy : 0.0;
    a.E[n] = make_float2(float(ex), float(ey));
    v[0] = ex * ex + ey * ey;
  }
  if (grid_sum<1>(v, a.part, a.ticket) && threadIdx.x == 0) a.fe[0] = 0.5 * v[0];
}

// --------------------------------------------------------------------------
// Multigrid V-cycle
// --------------------------------------------------------------------------
struct LevelDev {
  int nx, ny, nxn, nyn, px, py;
  float h2;
  const uint8_t *free;
  float *u, *f;
};

struct MGArgs {
  LevelDev L[16];
  int nlev;
  const PoissonState *ps;
};

// red-black Gauss-Seidel half sweep over one colour; zero_init: u starts at 0
__device__ __forceinline__ void smooth_node(const LevelDev &L, int n, int color, bool zero_init) {
  const int i = n / L.nyn, j = n - (n / L.nyn) * L.nyn;
  const bool mine = ((i + j) & 1) == color;
  if (!L.free[n]) {
    if (zero_init) L.u[n] = 0.f;
    return;
  }
  if (zero_init) {
    L.u[n] = mine ? 0.25f * L.h2 * L.f[n] : 0.f;
    return;
  }
  if (!mine) return;
  const int im = L.px ? wrapi(i - 1, L.nxn) : i - 1;
  const int ip = L.px ? wrapi(i + 1, L.nxn) : i + 1;
  const int jm = L.py ? wrapi(j - 1, L.nyn) : j - 1;
  const int jp = L.py ? wrapi(j + 1, L.nyn) : j + 1;
  const float s = L.h2 * L.f[n] + L.u[im * L.nyn + j] + L.u[ip * L.nyn + j] +
                  L.u[i * L.nyn + jm] + L.u[i * L.nyn + jp];
  L.u[n] = 0.25f * s;
}

__device__ __forceinline__ float resid_node(const LevelDev &L, int i, int j) {
  const int n = i * L.nyn + j;
  if (!L.free[n]) return 0.f;
  const int im = L.px ? wrapi(i - 1, L.nxn) : i - 1;
  const int ip = L.px ? wrapi(i + 1, L.nxn) : i + 1;
  const int jm = L.py ? wrapi(j - 1, L.nyn) : j - 1;
  const int jp = L.py ? wrapi(j + 1, L.nyn) : j + 1;
  const float Au = 4.f * L.u[n] - L.u[im * L.nyn + j] - L.u[ip * L.nyn + j] -
                   L.u[i * L.nyn + jm] - L.u[i * L.nyn + jp];
  return L.f[n] - Au / L.h2;
}

// full weighting of the fine residual onto coarse node nc
__device__ __forceinline__ void restrict_node(const LevelDev &F, const LevelDev &C, int nc) {
  if (!C.free[nc]) {
    C.f[nc] = 0.f;
    return;
  }
  const int I = nc / C.nyn, J = nc - (nc / C.nyn) * C.nyn;
  float s = 0.f;
#pragma unroll
  for (int a = -1; a <= 1; ++a) {
#pragma unroll
    for (int b = -1; b <= 1; ++b) {
      const int i = F.px ? wrapi(2 * I + a, F.nxn) : 2 * I + a;
      const int j = F.py ? wrapi(2 * J + b, F.nyn) : 2 * J + b;
      const float w = (a == 0 ? 2.f : 1.f) * (b == 0 ? 2.f : 1.f);
      s += w * resid_node(F, i, j);
    }
  }
  C.f[nc] = s * (1.f / 16.f);
}

// bilinear prolongation of the coarse correction, added on free fine nodes
__device__ __forceinline__ void prolong_node(const LevelDev &F, const LevelDev &C, int n) {
  if (!F.free[n]) return;
  const int i = n / F.nyn, j = n - (n / F.nyn) * F.nyn;
  const int I0 = i >> 1, J0 = j >> 1;
  const int I1 = (i & 1) ? (C.px ? wrapi(I0 + 1, C.nxn) : I0 + 1) : I0;
  const int J1 = (j & 1) ? (C.py ? wrapi(J0 + 1, C.nyn) : J0 + 1) : J0;
  float v;
  if (!(i & 1) && !(j & 1)) {
    v = C.u[I0 * C.nyn + J0];
  } else if (!(j & 1)) {
    v = 0.5f * (C.u[I0 * C.nyn + J0] + C.u[I1 * C.nyn + J0]);
  } else if (!(i & 1)) {
    v = 0.5f * (C.u[I0 * C.nyn + J0] + C.u[I0 * C.nyn + J1]);
  } else {
    v = 0.25f * (C.u[I0 * C.nyn + J0] + C.u[I1 * C.nyn + J0] + C.u[I0 * C.nyn + J1] +
                 C.u[I1 * C.nyn + J1]);
  }
  F.u[n] += v;
}

__global__ void k_smooth(MGArgs a, int l, int color, int zero_init) {
  if (a.ps->inner_done) return;
  const LevelDev &L = a.L[l];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < L.nxn * L.nyn) smooth_node(L, n, color, zero_init != 0);
}

__global__ void k_restrict(MGArgs a, int l) {
  if (a.ps->inner_done) return;
  const LevelDev &C = a.L[l + 1];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < C.nxn * C.nyn) restrict_node(a.L[l], C, n);
}

__global__ void k_prolong(MGArgs a, int l) {
  if (a.ps->inner_done) return;
  const LevelDev &F = a.L[l];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < F.nxn * F.nyn) prolong_node(F, a.L[l + 1], n);
}

// The V-cycle from level l0 to the coarsest, inside one CTA.
__global__ void __launch_bounds__(kCoarseThreads) k_coarse(MGArgs a, int l0) {
  if (a.ps->inner_done) return;
  const int last = a.nlev - 1;
  for (int l = l0; l <= last; ++l) {
    const LevelDev &L = a.L[l];
    const int nn = L.nxn * L.nyn;
    const int sweeps = (l == last) ? kCoarsestSweeps : 1;
    for (int k = threadIdx.x; k < nn; k += blockDim.x) smooth_node(L, k, 0, true);
    __syncthreads();
    for (int s = 0; s < sweeps; ++s) {
      if (s > 0) {
        for (int k = threadIdx.x; k < nn; k += blockDim.x) smooth_node(L, k, 0, false);
        __syncthreads();
      }
      for (int k = threadIdx.x; k < nn; k += blockDim.x) smooth_node(L, k, 1, false);
      __syncthreads();
    }
    if (l == last) {
      for (int s = 0; s < sweeps; ++s) {
        for (int k = threadIdx.x; k < nn; k += blockDim.x) smooth_node(L, k, 1, false);
        __syncthreads();
        for (int k = threadIdx.x; k < nn; k += blockDim.x) smooth_node(L, k, 0, false);
        __syncthreads();
      }
    } else {
      const LevelDev &C = a.L[l + 1];
      for (int k = threadIdx.x; k < C.nxn * C.nyn; k += blockDim.x) restrict_node(L, C, k);
      __syncthreads();
    }
  }
  for (int l = last - 1; l >= l0; --l) {
    const LevelDev &L = a.L[l];
    const int nn = L.nxn * L.nyn;
    for (int k = threadIdx.x; k < nn; k += blockDim.x) prolong_node(L, a.L[l + 1], k);
    __syncthreads();
    for (int k = threadIdx.x; k < nn; k += blockDim.x) smooth_node(L, k, 1, false);
    __syncthreads();
    for (int k = threadIdx.x; k < nn; k += blockDim.x) smooth_node(L, k, 0, false);
    __syncthreads();
  }
}

// --------------------------------------------------------------------------
FineArgs fine_args(pic_ctx *c) {
  FineArgs a;
  a.g = c->g;
  a.flags = c->d_nodeflags;
  a.lift = c->d_lift;
  a.gval = c->d_g;
  a.rho = c->d_rho;
  a.b = c->d_b;
  a.phi = c->d_phi;
  a.acc = c->d_acc;
  a.rho_ext = c->d_rho_ext;
  a.bottom = c->d_bottom;
  for (int s = 0; s < 2; ++s) {
    const double w = 1.0 / double(c->cfg.ppc[s]);
    a.qw[s] = c->cfg.charge[s] * w * std::ldexp(1.0, -kFracBits);
    a.sw[s] = c->cfg.charge[s] * w;
  }
  a.surface = c->cfg.surface_charge;
  a.r32 = c->d_r32;
  a.z = c->d_z;
  a.p_old = c->d_p0;
  a.p_new = c->d_p1;
  a.q = c->d_q;
  a.e = c->d_e;
  a.r64 = c->d_r64;
  a.ps = c->d_ps;
  a.part = c->red.part;
  a.ticket = c->red.ticket;
  a.singular = c->singular;
  a.rtol = c->cfg.poisson_rtol;
  a.maxit = c->cfg.poisson_maxit;
  a.step = c->d_step;
  a.advance_step = 0;
  a.E = c->d_E;
  a.fe = c->d_fe;
  return a;
}

MGArgs mg_args(pic_ctx *c) {
  MGArgs a;
  a.nlev = c->nlev;
  for (int l = 0; l < c->nlev; ++l) {
    const MGLevel &m = c->lev[l];
    a.L[l].nx = m.nx;
    a.L[l].ny = m.ny;
    a.L[l].nxn = m.nxn;
    a.L[l].nyn = m.nyn;
    a.L[l].px = c->g.px;
    a.L[l].py = c->g.py;
    a.L[l].h2 = m.h2;
    a.L[l].free = m.free;
    a.L[l].u = m.u;
    a.L[l].f = m.f;
  }
  a.ps = c->d_ps;
  return a;
}

inline int blocks_for(int n) { return (n + kThreads - 1) / kThreads; }

void launch_vcycle(pic_ctx *c, const MGArgs &a) {
  c->launches += 6 * c->lc + 1;
  for (int l = 0; l < c->lc; ++l) {
    const int nb = blocks_for(c->lev[l].nxn * c->lev[l].nyn);
    k_smooth<<<nb, kThreads, 0, c->stream>>>(a, l, 0, 1);
    k_smooth<<<nb, kThreads, 0, c->stream>>>(a, l, 1, 0);
    const int nbc = blocks_for(c->lev[l + 1].nxn * c->lev[l + 1].nyn);
    k_restrict<<<nbc, kThreads, 0, c->stream>>>(a, l);
  }
  k_coarse<<<1, kCoarseThreads, 0, c->stream>>>(a, c->lc);
  for (int l = c->lc - 1; l >= 0; --l) {
    const int nb = blocks_for(c->lev[l].nxn * c->lev[l].nyn);
    k_prolong<<<nb, kThreads, 0, c->stream>>>(a, l);
    k_smooth<<<nb, kThreads, 0, c->stream>>>(a, l, 1, 0);
    k_smooth<<<nb, kThreads, 0, c->stream>>>(a, l, 0, 0);
  }
}

}  // namespace

cudaError_t poisson_setup(pic_ctx *c) {
  const Geom &g = c->g;
  c->singular = 1;
  for (size_t n = 0; n < c->h_nodeflags.size(); ++n)
    if (!(c->h_nodeflags[n] & kFree)) c->singular = 0;
  // level hierarchy
  c->lev.clear();
  MGLevel L0;
  L0.nx = g.nx;
  L0.ny = g.ny;
  L0.nxn = g.nxn;
  L0.nyn = g.nyn;
  L0.h2 = 1.f;
  std::vector<std::vector<uint8_t>> masks;
  std::vector<uint8_t> m0(size_t(g.nxn) * g.nyn);
  for (size_t n = 0; n < m0.size(); ++n) m0[n] = (c->h_nodeflags[n] & kFree) ? 1 : 0;
  masks.push_back(m0);
  c->lev.push_back(L0);
  while (c->lev.size() < 16) {
    const MGLevel &F = c->lev.back();
    const bool even = (F.nx % 2 == 0) && (F.ny % 2 == 0);
    if (!even) break;
    const int cnx = F.nx / 2, cny = F.ny / 2;
    if (cnx < 2 || cny < 2) break;
    if (g.px && (cnx % 2)) break;
    if (g.py && (cny % 2)) break;
    MGLevel C;
    C.nx = cnx;
    C.ny = cny;
    C.nxn = g.px ? cnx : cnx + 1;
    C.nyn = g.py ? cny : cny + 1;
    C.h2 = F.h2 * 4.f;
    std::vector<uint8_t> mc(size_t(C.nxn) * C.nyn);
    const std::vector<uint8_t> &mf = masks.back();
    for (int I = 0; I < C.nxn; ++I)
      for (int J = 0; J < C.nyn; ++J) mc[size_t(I) * C.nyn + J] = mf[size_t(2 * I) * F.nyn + 2 * J];
    masks.push_back(mc);
    c->lev.push_back(C);
  }
  c->nlev = int(c->lev.size());
  c->lc = c->nlev - 1;
  for (int l = 0; l < c->nlev; ++l)
    if (c->lev[l].nxn * c->lev[l].nyn <= kSmallLevel) {
      c->lc = l;
      break;
    }
  const size_t nn = size_t(g.nxn) * g.nyn;
  for (int l = 0; l < c->nlev; ++l) {
    MGLevel &m = c->lev[l];
    const size_t n = size_t(m.nxn) * m.nyn;
    m.free = (uint8_t *)dev_alloc(c, n);
    if (!m.free) return cudaErrorMemoryAllocation;
    cudaMemcpy(m.free, masks[l].data(), n, cudaMemcpyHostToDevice);
    if (l == 0) {
      m.u = nullptr;
      m.f = nullptr;
    } else {
      m.u = (float *)dev_alloc(c, n * sizeof(float));
      m.f = (float *)dev_alloc(c, n * sizeof(float));
      if (!m.u || !m.f) return cudaErrorMemoryAllocation;
      cudaMemsetAsync(m.u, 0, n * sizeof(float), c->stream);
      cudaMemsetAsync(m.f, 0, n * sizeof(float), c->stream);
    }
  }
  float **vecs[] = {&c->d_r32, &c->d_z, &c->d_p0, &c->d_p1, &c->d_q, &c->d_e};
  for (float **v : vecs) {
    *v = (float *)dev_alloc(c, nn * sizeof(float));
    if (!*v) return cudaErrorMemoryAllocation;
    cudaMemsetAsync(*v, 0, nn * sizeof(float), c->stream);
  }
  c->lev[0].u = c->d_z;
  c->lev[0].f = c->d_r32;
  c->d_r64 = (double *)dev_alloc(c, nn * sizeof(double));
  c->red.nblocks = blocks_for(int(nn));
  c->red.part = (double *)dev_alloc(c, size_t(c->red.nblocks) * 4 * sizeof(double));
  c->red.ticket = (unsigned int *)dev_alloc(c, 64);
  c->d_ps = (PoissonState *)dev_alloc(c, sizeof(PoissonState));
  if (!c->d_r64 || !c->red.part || !c->red.ticket || !c->d_ps) return cudaErrorMemoryAllocation;
  cudaMemsetAsync(c->red.ticket, 0, 64, c->stream);
  cudaMemsetAsync(c->d_ps, 0, sizeof(PoissonState), c->stream);
  cudaError_t e = cudaMallocHost((void **)&c->h_ps, sizeof(PoissonState));
  if (e != cudaSuccess) return e;
  cudaEventCreate(&c->ev0);
  cudaEventCreate(&c->ev1);
  return cudaGetLastError();
}

cudaError_t launch_rho(pic_ctx *c, int advance_step) {
  FineArgs a = fine_args(c);
  a.advance_step = advance_step;
  const int nn = c->g.nxn * c->g.nyn;
  k_rho<<<blocks_for(nn), kThreads, 0, c->stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_field(pic_ctx *c) {
  FineArgs a = fine_args(c);
  const int nn = c->g.nxn * c->g.nyn;
  k_field<<<blocks_for(nn), kThreads, 0, c->stream>>>(a);
  return cudaGetLastError();
}

pic_status poisson_solve(pic_ctx *c, bool zero_guess) {
  FineArgs a = fine_args(c);
  const MGArgs m = mg_args(c);
  const int nn = c->g.nxn * c->g.nyn;
  const int nb = blocks_for(nn);
  cudaEventRecord(c->ev0, c->stream);
  if (zero_guess) k_phi_reset<<<nb, kThreads, 0, c->stream>>>(a);
  cudaMemsetAsync(&c->d_ps->total_iters, 0, sizeof(int32_t), c->stream);
  int outer = 0;
  const int batch = 4;
  bool converged = false;
  if (zero_guess) c->launches += 1;
  for (; outer < kMaxOuter + 1; ++outer) {
    k_resid64<<<nb, kThreads, 0, c->stream>>>(a);
    c->launches += 1;
    cudaMemcpyAsync(c->h_ps, c->d_ps, sizeof(PoissonState), cudaMemcpyDeviceToHost, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return PIC_ECUDA;
    if (c->h_ps->outer_done) {
      converged = true;
      break;
    }
    if (outer == kMaxOuter) break;
    launch_vcycle(c, m);
    k_rz<<<nb, kThreads, 0, c->stream>>>(a);
    c->launches += 1;
    for (int it = 0; it < c->cfg.poisson_maxit; it += batch) {
      for (int b = 0; b < batch; ++b) {
        k_pq<<<nb, kThreads, 0, c->stream>>>(a);
        k_update<<<nb, kThreads, 0, c->stream>>>(a);
        launch_vcycle(c, m);
        k_rz<<<nb, kThreads, 0, c->stream>>>(a);
        c->launches += 3;
      }
      cudaMemcpyAsync(c->h_ps, c->d_ps, sizeof(PoissonState), cudaMemcpyDeviceToHost, c->stream);
      if (cudaStreamSynchronize(c->stream) != cudaSuccess) return PIC_ECUDA;
      if (c->h_ps->inner_done) break;
    }
    k_correct<<<nb, kThreads, 0, c->stream>>>(a);
    c->launches += 1;
  }
  cudaEventRecord(c->ev1, c->stream);
  cudaMemcpyAsync(c->h_ps, c->d_ps, sizeof(PoissonState), cudaMemcpyDeviceToHost, c->stream);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return PIC_ECUDA;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  c->last_ms = ms;
  c->last_outer = outer;
  if (cudaGetLastError() != cudaSuccess) return PIC_ECUDA;
  if (!converged) {
    k_set_status<<<1, 1, 0, c->stream>>>(c->d_status, PIC_ST_NOCONV);
    return PIC_ENOCONV;
  }
  return PIC_OK;
}

}  // namespace picgb
