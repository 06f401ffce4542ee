// 3x3 convolutions of the warm-start U-Net on the fifth-generation tensor
// cores: an implicit GEMM whose products run as tcgen05.mma with the FP32
// accumulator in tensor memory (TMEM), operands staged in shared memory by
// the tensor memory accelerator (TMA).
//
// out[b][h][w][n] = act(bias[n] + sum_{dy,dx,c} in[b][h+dy-1][w+dx-1][c] W[n][3 dy + dx][c])
// with BF16 tensors in NHWC (channel slices given by a channel stride and
// offset), FP32 accumulation, act = ReLU or identity, zero padding.
//
// One CTA computes a tile of M = 128 output pixels (a BH x BW block of one
// image, BW = min(W, 128) rounded down to a power of two) for a block of N
// output channels: all of them, or, for layers with fewer pixel tiles than
// SMs, one of the column blocks that the grid's second index selects.  The
// K loop runs over the 9 taps times cin / KB channel blocks.  For each block
// a 4-D TMA box {KB channels, BW, BH, 1} of the input,
// shifted by the tap, lands in shared memory in the swizzled K-major layout
// the MMA reads (zero fill supplies the padding), and a 2-D box {KB, N} of
// the weights [cout][9][cin] beside it.  Warp 0 lane 0 issues the TMA loads
// into a ring of stages (mbarrier expect-tx), warp 1 lane 0 issues KB / 16
// MMAs of 128 x N x 16 per stage and releases the stage by tcgen05.commit;
// then all four warps read their 32 TMEM lanes (one pixel per thread),
// add the bias, apply the activation and store BF16.  Every wait is bounded:
// a wait that gives up sets the error word and the CTA winds down (releasing
// its TMEM) instead of hanging.
//
// The same kernel, in further modes, computes the 2x2 stride-2 transposed
// convolution and its data gradient; k_wgrad_tc below computes the weight
// gradients of both kinds of convolution with both operands MN-major.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "internal.cuh"

namespace picgb {
namespace tc {

typedef __nv_bfloat16 bf16;

constexpr int kM = 128;            // output pixels per CTA = TMEM lanes
constexpr int kThreads = 128;      // four warps
constexpr uint64_t kWaitNs = 2000000000ull;   // a wait gives up after 2 s (globaltimer)

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t saddr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// wait for the phase of the given parity to complete, giving up after kWaitNs
// of wall time (one poll may itself suspend for a while, so the number of
// polls alone would not bound the time)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = gtime();
  do {
    if (mbar_try(bar, parity)) return true;
  } while (gtime() - t0 < kWaitNs);
  return false;
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            int c3, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            int c3, int c4, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D[tmem] (+)= A[smem] . B[smem]^T, M = 128, N from the instruction descriptor, K = 16
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrives on the mbarrier once every MMA this thread issued before has completed
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
// 32 lanes x 16 consecutive 32-bit columns: register k of lane l = TMEM[lane base + l][col + k]
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile in the swizzled
// layout TMA wrote: start address, the (unused) leading byte offset, the
// stride between groups of 8 rows (8 x row bytes), the descriptor version of
// this architecture, and the swizzle mode (2: 128 B, 4: 64 B, 6: 32 B rows).
template <int KB>
struct Swz {
  static constexpr uint32_t row_bytes = KB * 2;
  static constexpr uint64_t layout = KB == 64 ? 2 : (KB == 32 ? 4 : 6);
};
template <int KB>
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return uint64_t((addr & 0x3FFFF) >> 4) | (uint64_t(1) << 16) |
         (uint64_t((8 * Swz<KB>::row_bytes) >> 4) << 32) | (uint64_t(1) << 46) | (Swz<KB>::layout << 61);
}
// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N / 8 and M / 16.
template <int N>
__host__ __device__ constexpr uint32_t instr_desc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(kM >> 4) << 24);
}

struct TCArgs {
  bf16 *out;
  int out_cs, out_off;
  const float *bias;   // [cout] or null
  int relu;
  int B, H, W, cin, in_off;
  int BW, BH, tiles_w, tiles_h;
  int n_base;          // first GEMM column of this launch; CTA row y of the grid adds y N
  int up_cout;         // transposed convolution: output channels (GEMM column n = (2a + c) up_cout + co)
  int ncols;           // data gradient of the transposed convolution: GEMM columns (weight rows per tap)
  int *err;            // error word: 1 producer, 2 MMA, 3 epilogue wait gave up
};

constexpr int kHaloPix = kM + 2;   // one image row of the tile and its two neighbours

// Shared memory of one CTA: STAGES A stages, then STAGES B stages, then the
// barriers.  Per stage, A is the 128 x KB input tile of one tap, or (HALO) the
// 130 x KB input row of one vertical tap, and B is the N x KB weight tile of
// one tap, or (HALO) the three horizontal taps' tiles side by side.
template <int N, int KB, int STAGES, bool HALO = false>
struct Layout {
  static constexpr uint32_t B_TILE = N * KB * 2;
  static constexpr uint32_t A_BYTES = HALO ? ((kHaloPix * KB * 2 + 1023) / 1024) * 1024 : kM * KB * 2;
  static constexpr uint32_t A_TX = HALO ? kHaloPix * KB * 2 : kM * KB * 2;   // bytes TMA writes
  static constexpr uint32_t B_BYTES = (HALO ? 3 : 1) * B_TILE;
  static constexpr uint32_t BAR_OFF = STAGES * (A_BYTES + B_BYTES);
  static constexpr uint32_t BYTES = BAR_OFF + (2 * STAGES + 1) * 8 + 16 + 1024;   // + alignment slack
  static constexpr uint32_t NCOLS = N < 32 ? 32 : N;
};

// UP: the 2x2 stride-2 transposed convolution instead of the 3x3 one -- one
// tap (the input pixel itself), GEMM columns n = (2a + c) up_cout + co, and
// the result of input pixel (y, x) written to output pixel (2y + a, 2x + c).
// HALO (tiles of one image row, BW = 128): the K loop runs over the three
// vertical taps times the channel blocks; each step loads the 130-pixel input
// row once and the three horizontal taps read it from rows 0, 1, 2 -- the
// MMA's start address moves by whole swizzled rows, and the swizzle follows
// the shared-memory address, so the shifted operand is the tap's tile.  That
// moves a third of the input bytes of nine shifted tiles.
// UPB: the data gradient of the transposed convolution.  Input pixel (y, x)
// of that convolution gathers, over its four children (2y + a, 2x + c), the
// output gradient's channels: four taps t = 2a + c, each a 5-D box {KB, 1,
// BW, 1, BH} of the gradient viewed as {channels, c, x, a, image rows} -- the
// rows of the tap's 128 pixels, in the same K-major layout as the other
// modes.  B: the weights [4 ncols][cout], rows t ncols + n.
template <int N, int KB, int STAGES, bool UP, bool HALO = false, bool UPB = false>
__global__ void __launch_bounds__(kThreads, 1)
    k_conv3x3_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TCArgs a) {
  static_assert(!(UP && HALO), "the transposed convolution has one tap");
  static_assert(!(UPB && (UP || HALO)), "one mode at a time");
  using L = Layout<N, KB, STAGES, HALO>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sA = saddr(smem), sB = sA + STAGES * L::A_BYTES;
  const uint32_t bar0 = sA + L::BAR_OFF;           // full[s] = bar0 + 8 s, empty[s] = bar0 + 8 (STAGES + s)
  const uint32_t done = bar0 + 16 * STAGES;
  uint32_t *slot = reinterpret_cast<uint32_t *>(smem + L::BAR_OFF + (2 * STAGES + 1) * 8);
  __shared__ int s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int t = blockIdx.x;
  const int tw = t % a.tiles_w;
  t /= a.tiles_w;
  const int th = t % a.tiles_h;
  const int b = t / a.tiles_h;
  const int w0 = tw * a.BW, h0 = th * a.BH;
  const int nb0 = a.n_base + int(blockIdx.y) * N;   // this CTA's first GEMM column

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(bar0 + 8 * s, 1);
      mbar_init(bar0 + 8 * (STAGES + s), 1);
    }
    mbar_init(done, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(saddr(slot), L::NCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  const int kchunks = a.cin / KB;
  const int nk = (UP ? 1 : (HALO ? 3 : (UPB ? 4 : 9))) * kchunks;

  if (tid == 0) {
    // TMA producer: stage s of round r is reused once the MMAs of round r - 1 released it
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (kb / STAGES) & 1;
      if (kb >= STAGES && !mbar_wait(bar0 + 8 * (STAGES + s), ph ^ 1)) {
        atomicExch(&s_fail, 1);
        atomicCAS(a.err, 0, 1);
        break;
      }
      if (s_fail) break;
      if (UPB) {
        const int tap = kb / kchunks, c0 = (kb - tap * kchunks) * KB;
        mbar_expect_tx(bar0 + 8 * s, L::A_TX + L::B_BYTES);
        tma_load_5d(sA + s * L::A_BYTES, &tmA, a.in_off + c0, tap & 1, w0, tap >> 1, b * a.H + h0, bar0 + 8 * s);
        tma_load_2d(sB + s * L::B_BYTES, &tmB, c0, tap * a.ncols + nb0, bar0 + 8 * s);
        continue;
      }
      if (HALO) {
        const int dy = kb / kchunks, c0 = (kb - dy * kchunks) * KB;
        mbar_expect_tx(bar0 + 8 * s, L::A_TX + L::B_BYTES);
        tma_load_4d(sA + s * L::A_BYTES, &tmA, a.in_off + c0, w0 - 1, h0 + dy - 1, b, bar0 + 8 * s);
        for (int dx = 0; dx < 3; ++dx)
          tma_load_2d(sB + s * L::B_BYTES + dx * L::B_TILE, &tmB, (3 * dy + dx) * a.cin + c0, nb0, bar0 + 8 * s);
        continue;
      }
      const int tap = UP ? 4 : kb / kchunks, c0 = (kb - (UP ? 0 : tap) * kchunks) * KB;
      const int dy = tap / 3 - 1, dx = tap - 3 * (tap / 3) - 1;
      mbar_expect_tx(bar0 + 8 * s, L::A_TX + L::B_BYTES);
      tma_load_4d(sA + s * L::A_BYTES, &tmA, a.in_off + c0, w0 + dx, h0 + dy, b, bar0 + 8 * s);
      if (UP)
        tma_load_2d(sB + s * L::B_BYTES, &tmB, c0, nb0, bar0 + 8 * s);
      else
        tma_load_2d(sB + s * L::B_BYTES, &tmB, tap * a.cin + c0, nb0, bar0 + 8 * s);
    }
  } else if (tid == 32) {
    // MMA issuer
    constexpr uint32_t idesc = instr_desc<N>();
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (kb / STAGES) & 1;
      if (!mbar_wait(bar0 + 8 * s, ph)) {
        atomicExch(&s_fail, 1);
        atomicCAS(a.err, 0, 2);
        break;
      }
      tc_fence_after();
      if (HALO) {
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          const uint64_t da = smem_desc<KB>(sA + s * L::A_BYTES + dx * Swz<KB>::row_bytes);   // row dx on
          const uint64_t db = smem_desc<KB>(sB + s * L::B_BYTES + dx * L::B_TILE);
#pragma unroll
          for (int k = 0; k < KB / 16; ++k)
            mma_bf16(tmem, da + 2 * k, db + 2 * k, idesc, (kb | dx | k) != 0 ? 1u : 0u);
        }
      } else {
        const uint64_t da = smem_desc<KB>(sA + s * L::A_BYTES);
        const uint64_t db = smem_desc<KB>(sB + s * L::B_BYTES);
#pragma unroll
        for (int k = 0; k < KB / 16; ++k)   // 16 elements = 32 bytes along the swizzled row
          mma_bf16(tmem, da + 2 * k, db + 2 * k, idesc, (kb | k) != 0 ? 1u : 0u);
      }
      mma_commit(bar0 + 8 * (STAGES + s));
    }
    mma_commit(done);
  }

  // epilogue: thread (warp w, lane l) owns pixel 32 w + l, the accumulator's TMEM lane
  __syncwarp();
  const bool ok = mbar_wait(done, 0);
  tc_fence_after();
  if (!ok) atomicCAS(a.err, 0, 3);
  const int p = 32 * warp + lane;
  const int h = h0 + p / a.BW, w = w0 + p % a.BW;
  const bool inside = h < a.H && w < a.W;
  const uint32_t tl = tmem + (uint32_t(32 * warp) << 16);
#pragma unroll 1
  for (int n0 = 0; n0 < N; n0 += 16) {
    uint32_t r[16];
    tmem_ld16(tl + n0, r);
    if (ok && !s_fail && inside) {
      // destination and bias of these 16 columns (16 divides up_cout: one (a, c) per chunk)
      bf16 *dst;
      int co;
      if (UP) {
        const int n = nb0 + n0, ac = n / a.up_cout;
        co = n - ac * a.up_cout;
        const int oh = 2 * h + (ac >> 1), ow = 2 * w + (ac & 1);
        dst = a.out + ((size_t(b) * 2 * a.H + oh) * 2 * a.W + ow) * a.out_cs + a.out_off + co;
      } else {
        co = nb0 + n0;
        dst = a.out + ((size_t(b) * a.H + h) * a.W + w) * a.out_cs + a.out_off + co;
      }
      __align__(16) bf16 o[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        float v = __uint_as_float(r[k]) + (a.bias ? __ldg(a.bias + co + k) : 0.f);
        if (a.relu) v = fmaxf(v, 0.f);
        o[k] = __float2bfloat16_rn(v);
      }
      reinterpret_cast<uint4 *>(dst)[0] = reinterpret_cast<const uint4 *>(o)[0];
      reinterpret_cast<uint4 *>(dst)[1] = reinterpret_cast<const uint4 *>(o)[1];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, L::NCOLS);
}

// ---------------------------------------------------------------- first layer
// The network's first 3x3 convolution (2 input channels -> 32) on the tensor
// cores.  The 9 taps x 2 channels of a pixel, BF16-rounded, form one K row of
// 32 (k = 2 tap + c, zeros from 18 on) of an A tile that the threads write to
// shared memory, in the non-swizzled K-major layout: core matrices of 8 rows
// x 16 bytes, 8 K values per plane of 128 rows, planes LBO = 2048 B apart,
// 8-row groups SBO = 128 B apart.  B, the 32 x 32 weight matrix, has the same
// layout (planes of 32 rows).  A CTA takes tiles of 128 consecutive pixels
// (row-major over images, rows and columns) in turn: the threads build A,
// one thread issues two MMAs of K = 16 into the TMEM accumulator and commits,
// and the four warps read their 32 lanes back (bias, activation, BF16).
constexpr int kInCh = 2, kInK = 32, kInN = 32;

__device__ __forceinline__ uint64_t plain_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((addr & 0x3FFFF) >> 4) | (uint64_t(lbo >> 4) << 16) | (uint64_t(sbo >> 4) << 32) |
         (uint64_t(1) << 46);   // layout type 0: no swizzle
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const uint32_t a = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
  const uint32_t b = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
  return a | (b << 16);
}

__global__ void __launch_bounds__(kThreads, 1)
    k_conv_in_tc(const float2 *x, const bf16 *w, int wcin, const float *bias, bf16 *out, int B, int H, int W,
                 int relu, int *err) {
  __shared__ __align__(1024) uint8_t sA[(kInK / 8) * kM * 16];     // 4 planes of 128 rows
  __shared__ __align__(1024) uint8_t sB[(kInK / 8) * kInN * 16];   // 4 planes of 32 rows
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t slot;
  __shared__ float sbias[kInN];
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // B[n][k] = w[n][tap][c], k = 2 tap + c < 18, else 0
  for (int i = tid; i < kInN * kInK; i += kThreads) {
    const int n = i / kInK, k = i - (i / kInK) * kInK;
    const bf16 v = k < 9 * kInCh ? w[(size_t(n) * 9 + k / kInCh) * wcin + (k % kInCh)] : __float2bfloat16(0.f);
    *reinterpret_cast<bf16 *>(sB + (k / 8) * (kInN * 16) + n * 16 + (k % 8) * 2) = v;
  }
  for (int i = tid; i < kInN; i += kThreads) sbias[i] = bias ? bias[i] : 0.f;
  if (tid == 0) {
    mbar_init(saddr(&bar), 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(saddr(&slot), kInN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = slot;
  constexpr uint32_t idesc = instr_desc<kInN>();
  const unsigned npix = unsigned(B) * unsigned(H) * unsigned(W);
  const unsigned ntiles = (npix + kM - 1) / kM;
  uint32_t it = 0;
  for (unsigned tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    // this thread's pixel (the A row tid) and its 9 x 2 inputs, zeros outside
    // the image or past the end
    const unsigned p = tile * kM + unsigned(tid);
    const bool valid = p < npix;
    const unsigned r = valid ? p / unsigned(W) : 0u;
    const int wq = valid ? int(p - r * unsigned(W)) : 0;
    const int h = int(r % unsigned(H));
    float v[2 * 9];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int hh = h + t / 3 - 1, ww = wq + t % 3 - 1;
      float2 e = make_float2(0.f, 0.f);
      if (valid && hh >= 0 && hh < H && ww >= 0 && ww < W) e = x[int(p) + (t / 3 - 1) * W + (t % 3 - 1)];
      v[2 * t] = e.x;
      v[2 * t + 1] = e.y;
    }
    const uint4 q0 = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
    const uint4 q1 = make_uint4(pack_bf16(v[8], v[9]), pack_bf16(v[10], v[11]), pack_bf16(v[12], v[13]),
                                pack_bf16(v[14], v[15]));
    const uint4 q2 = make_uint4(pack_bf16(v[16], v[17]), 0u, 0u, 0u);
    const uint4 q3 = make_uint4(0u, 0u, 0u, 0u);
    reinterpret_cast<uint4 *>(sA + 0 * kM * 16)[tid] = q0;
    reinterpret_cast<uint4 *>(sA + 1 * kM * 16)[tid] = q1;
    reinterpret_cast<uint4 *>(sA + 2 * kM * 16)[tid] = q2;
    reinterpret_cast<uint4 *>(sA + 3 * kM * 16)[tid] = q3;
    fence_async_smem();   // the threads' writes become visible to the tensor core's reads
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int k = 0; k < kInK / 16; ++k)   // planes 2k, 2k + 1
        mma_bf16(tmem, plain_desc(saddr(sA) + 2 * k * (kM * 16), kM * 16, 128),
                 plain_desc(saddr(sB) + 2 * k * (kInN * 16), kInN * 16, 128), idesc, k ? 1u : 0u);
      mma_commit(saddr(&bar));
    }
    __syncwarp();
    const bool ok = __all_sync(0xffffffffu, mbar_wait(saddr(&bar), it & 1));
    tc_fence_after();
    if (ok) {
      const uint32_t tl = tmem + (uint32_t(32 * warp) << 16);
#pragma unroll
      for (int n0 = 0; n0 < kInN; n0 += 16) {
        uint32_t rr[16];
        tmem_ld16(tl + n0, rr);
        if (valid) {
          __align__(16) bf16 o[16];
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            float y = __uint_as_float(rr[k]) + sbias[n0 + k];
            if (relu) y = fmaxf(y, 0.f);
            o[k] = __float2bfloat16_rn(y);
          }
          uint4 *dst = reinterpret_cast<uint4 *>(out + size_t(p) * kInN + n0);
          dst[0] = reinterpret_cast<const uint4 *>(o)[0];
          dst[1] = reinterpret_cast<const uint4 *>(o)[1];
        }
      }
    } else if (lane == 0) {
      atomicExch(&s_fail, 1);
      atomicCAS(err, 0, 3);
    }
    tc_fence_before();
    __syncthreads();   // TMEM read and A free for the next tile
    if (s_fail) break;
  }
  if (warp == 0) tmem_dealloc(tmem, kInN);
}

// ---------------------------------------------------------------- weight gradient
// dW[co][3 dy + dx][ci] += sum_p dpre[p][co] in[p + (dy - 1, dx - 1)][ci] (zero
// padding), dpre the gradient before the ReLU [B][H][W][cout], in the layer's
// input.  A K block is KP = 64 consecutive pixels (w0 .. w0 + 63) of one input
// row hq of one image.  Both operands are MN-major: pixels (K) are the rows
// of a swizzled tile, channels (M, N) run along the row.
//  * B, the input: the row hq from pixel w0 - 8 to w0 + KP + 7 (TMA box
//    {CI, KP + 16}; the x coordinate stays a multiple of 8), CI channels.
//    The three horizontal taps are three N chunks of CI channels whose
//    starts lie one pixel row apart (LBO = one row), so N = 3 CI covers
//    dx = 0, 1, 2 at once, each chunk being the input shifted by dx - 1.
//  * A, the gradient: three slots, slot s the dpre row hq + 1 - s (pixels w0
//    .. w0 + KP - 1, zero fill off the image), one slot per vertical tap
//    (dpre row hq + 1 - dy meets input row hq at tap dy), and a fourth slot
//    of zeros.  M = 128 rows of D are slots of CO channels at LBO = one slot:
//    CO = 32, all four slots in one MMA; CO = 64, slots {0, 1} and {2, 3}.
// D row (s, co), column (dx, ci) thus accumulates dW[co][3 s + dx][ci] over
// the CTA's K blocks; the epilogue adds it to dW with vector atomics (FP32,
// so the sum order, not the terms, depends on the grid).
// UPW: the weight gradient of the 2x2 stride-2 transposed convolution,
// dW[a][c][ci][co] = sum over input pixels p of in[p][ci] g[child (a, c) of p][co],
// g its output gradient.  The four slots of A are the four children's tiles
// of g (5-D boxes {CO, 1, 64, 1, 1} of g viewed as {channels, c, x, a, rows}),
// B is the input row without a shift (N = CI), and D row (t, co), column ci
// holds dW[t][ci][co]; the epilogue adds it with scalar atomics, consecutive
// lanes on consecutive co.
constexpr int kWKP = 64;   // pixels per K block

template <int CO, int CI, int STAGES, bool UPW = false>
struct WLayout {
  static constexpr int KPB = kWKP + 16;   // the input row with 8-pixel margins
  static constexpr uint32_t SLOT = kWKP * CO * 2;
  static constexpr uint32_t A_BYTES = 4 * SLOT;
  static constexpr uint32_t B_TX = KPB * CI * 2;
  static constexpr uint32_t B_BYTES = ((B_TX + 1023) / 1024) * 1024;
  static constexpr uint32_t STAGE = A_BYTES + B_BYTES;
  static constexpr uint32_t BAR_OFF = STAGES * STAGE;
  // allocated, never written: keeps every address the descriptors of the last
  // stage can form inside this CTA's shared memory (the widest reading of
  // the B tile spans 3 CI rows of 8-row groups from row 55)
  static constexpr uint32_t TAIL = 6 * CI * CI + 112 * CI;
  static constexpr uint32_t BYTES = BAR_OFF + (2 * STAGES + 1) * 8 + 16 + TAIL + 1024;
  static constexpr int NM = CO == 32 ? 1 : 2;   // MMAs along M per 16 pixels
  static constexpr int N = UPW ? CI : 3 * CI;
  static constexpr uint32_t NCOLS = NM * N <= 32 ? 32 : NM * N <= 64 ? 64 : NM * N <= 128 ? 128 : NM * N <= 256 ? 256 : 512;
};

// descriptor of an MN-major tile in the swizzled layout TMA wrote with rows
// of CH channels: K rows CH x 2 bytes apart, groups of 8 rows SBO = 8 rows
// apart, chunks of CH channels along M or N at LBO
template <int CH>
__device__ __forceinline__ uint64_t mn_desc(uint32_t addr, uint32_t lbo) {
  return uint64_t((addr & 0x3FFFF) >> 4) | (uint64_t(lbo >> 4) << 16) |
         (uint64_t((8 * Swz<CH>::row_bytes) >> 4) << 32) | (uint64_t(1) << 46) | (Swz<CH>::layout << 61);
}
// kind::f16 with BF16 A and B, both MN-major (transpose bits 15 and 16)
template <int N>
__host__ __device__ constexpr uint32_t instr_desc_mn() {
  return instr_desc<N>() | (1u << 15) | (1u << 16);
}

struct WArgs {
  float *dw;           // [cout][9][cin]; UPW: [4][cin][cout]
  int cin, cout, in_off, a_off, H, nwc;
  long long nkb;       // K blocks: B H rows x nwc pixel chunks
  long long per_cta;   // K blocks per CTA along the grid's first index
  int *err;
};

template <int CO, int CI, int STAGES, bool UPW = false>
__global__ void __launch_bounds__(kThreads, 1)
    k_wgrad_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, WArgs a) {
  using L = WLayout<CO, CI, STAGES, UPW>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t s0 = saddr(smem);
  const uint32_t bar0 = s0 + L::BAR_OFF;   // full[s] = bar0 + 8 s, empty[s] = bar0 + 8 (STAGES + s)
  const uint32_t done = bar0 + 16 * STAGES;
  uint32_t *slot = reinterpret_cast<uint32_t *>(smem + L::BAR_OFF + (2 * STAGES + 1) * 8);
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ncib = a.cin / CI;
  const int co0 = int(blockIdx.y) / ncib * CO, ci0 = int(blockIdx.y) % ncib * CI;
  const long long k0 = blockIdx.x * a.per_cta;
  const long long k1 = k0 + a.per_cta < a.nkb ? k0 + a.per_cta : a.nkb;
  const int nk = int(k1 - k0);   // at least 1 (the host sizes the grid so)

  // the fourth A slot of every stage holds zeros (the MMA's rows 96..127 for
  // CO = 32, 64..127 of the second MMA for CO = 64; discarded)
  if (!UPW) {
    for (int st = 0; st < STAGES; ++st)
      for (uint32_t o = 16 * tid; o < L::SLOT; o += 16 * kThreads)
        *reinterpret_cast<uint4 *>(smem + st * L::STAGE + 3 * L::SLOT + o) = make_uint4(0, 0, 0, 0);
    fence_async_smem();
  }
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(bar0 + 8 * s, 1);
      mbar_init(bar0 + 8 * (STAGES + s), 1);
    }
    mbar_init(done, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(saddr(slot), L::NCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;

  if (tid == 0) {
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (kb / STAGES) & 1;
      if (kb >= STAGES && !mbar_wait(bar0 + 8 * (STAGES + s), ph ^ 1)) {
        atomicExch(&s_fail, 1);
        atomicCAS(a.err, 0, 1);
        break;
      }
      if (s_fail) break;
      const long long g = k0 + kb;
      const long long r = g / a.nwc;              // b H + hq
      const int w0 = int(g - r * a.nwc) * kWKP;
      const int b = int(r / a.H), hq = int(r - (long long)b * a.H);
      const uint32_t st = s0 + s * L::STAGE;
      mbar_expect_tx(bar0 + 8 * s, (UPW ? 4 : 3) * L::SLOT + L::B_TX);
      if (UPW) {
        for (int t = 0; t < 4; ++t)
          tma_load_5d(st + t * L::SLOT, &tmA, a.a_off + co0, t & 1, w0, t >> 1, int(r), bar0 + 8 * s);
      } else {
        for (int sl = 0; sl < 3; ++sl)
          tma_load_4d(st + sl * L::SLOT, &tmA, co0, w0, hq + 1 - sl, b, bar0 + 8 * s);
      }
      tma_load_4d(st + L::A_BYTES, &tmB, a.in_off + ci0, w0 - 8, hq, b, bar0 + 8 * s);
    }
  } else if (tid == 32) {
    constexpr uint32_t idesc = instr_desc_mn<L::N>();
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (kb / STAGES) & 1;
      if (!mbar_wait(bar0 + 8 * s, ph)) {
        atomicExch(&s_fail, 1);
        atomicCAS(a.err, 0, 2);
        break;
      }
      tc_fence_after();
      const uint32_t st = s0 + s * L::STAGE;
#pragma unroll
      for (int k = 0; k < kWKP / 16; ++k) {
        // input rows 7 + 16 k ..: pixel w0 - 1 + 16 k on, the tap dx = 0 chunk
        // (UPW: rows 8 + 16 k .., pixel w0 + 16 k on)
        const uint64_t db = mn_desc<CI>(st + L::A_BYTES + ((UPW ? 8 : 7) + 16 * k) * (CI * 2), CI * 2);
#pragma unroll
        for (int m = 0; m < L::NM; ++m) {
          const uint64_t da = mn_desc<CO>(st + 2 * m * L::SLOT + 16 * k * (CO * 2), L::SLOT);
          mma_bf16(tmem + m * L::N, da, db, idesc, (kb | k) != 0 ? 1u : 0u);
        }
      }
      mma_commit(bar0 + 8 * (STAGES + s));
    }
    mma_commit(done);
  }

  // epilogue: warp w reads D rows 32 w .. 32 w + 31 of each accumulator
  __syncwarp();
  const bool ok = mbar_wait(done, 0);
  tc_fence_after();
  if (!ok) atomicCAS(a.err, 0, 3);
#pragma unroll
  for (int m = 0; m < L::NM; ++m) {
    const int row = 32 * warp + lane;                       // D row of MMA m
    const int sl = CO == 32 ? warp : 2 * m + (row >> 6);    // A slot: vertical tap (UPW: child)
    const int co = co0 + (CO == 32 ? lane : (row & 63));
    if (!UPW && sl == 3) continue;                          // warp-uniform: the zero slot
    const uint32_t tl = tmem + (uint32_t(32 * warp) << 16) + m * L::N;
#pragma unroll 1
    for (int n0 = 0; n0 < L::N; n0 += 16) {
      uint32_t v[16];
      tmem_ld16(tl + n0, v);
      if (UPW) {
        // consecutive lanes: consecutive co of one (t, ci) row of dW
        if (ok && !s_fail) {
          float *dst = a.dw + (size_t(sl) * a.cin + ci0 + n0) * a.cout + co;
#pragma unroll
          for (int q = 0; q < 16; ++q) atomicAdd(dst + size_t(q) * a.cout, __uint_as_float(v[q]));
        }
      } else if (ok && !s_fail) {
        const int dx = n0 / CI, ci = ci0 + (n0 - dx * CI);
        float4 *dst = reinterpret_cast<float4 *>(a.dw + (size_t(co) * 9 + 3 * sl + dx) * a.cin + ci);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          atomicAdd(dst + q, make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                         __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3])));
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, L::NCOLS);
}

// ---------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

CUtensorMapSwizzle swizzle_of(int kb) {
  return kb == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : (kb == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
}

// Launch shape, from timings of the network's layers at 1032 x 512 (the
// results do not depend on it, bit for bit):
//  * column blocks: a layer with fewer pixel tiles than SMs splits its N
//    columns into blocks of N / 2, N / 4 (no narrower than 64), one per CTA
//    row of the grid (N 256 over 65 tiles: 22.7 us -> 18.6 us as 4 x 64);
//  * ring depth: the deepest ring (4, 3 or 2 stages) whose CTAs all fit on
//    the SMs at once; when no depth gives one wave, the depth that leaves
//    the most CTAs per SM, because more resident CTAs hide the TMA round
//    trips better than a deeper ring (N 32, KB 64: 51 us with 2 stages, 74 us
//    with 4; N 128, KB 64 over 258 tiles: 12.4 us with 3, 16.6 us with 4).
// The depth is chosen at run time for KB = 64; KB = 16 and 32 (the wide
// top level only) take one tabled depth.
constexpr uint32_t kSmemPerSm = 233472;   // shared memory of an SM for CTAs
constexpr uint32_t kSmemPerCta = 1024;    // reserved by the system per CTA

template <int N, int KB>
constexpr int stages_of() {
  return KB == 16 ? 4 : (KB == 32 ? 3 : 2);
}

// resident CTAs per SM of an instantiation: shared memory, TMEM columns, threads
template <int N, int KB, int STAGES>
constexpr int occupancy_of() {
  constexpr int by_smem = int(kSmemPerSm / (Layout<N, KB, STAGES>::BYTES + kSmemPerCta));
  constexpr int by_tmem = int(512 / Layout<N, KB, STAGES>::NCOLS);
  constexpr int by_threads = 2048 / kThreads;
  return by_smem < by_tmem ? (by_smem < by_threads ? by_smem : by_threads)
                           : (by_tmem < by_threads ? by_tmem : by_threads);
}

// the dynamic shared memory size of one instantiation (set once per process,
// before any stream capture)
template <int N, int KB, int STAGES, bool UP, bool HALO = false>
cudaError_t prepare_nks() {
  static cudaError_t e = cudaFuncSetAttribute(k_conv3x3_tc<N, KB, STAGES, UP, HALO>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              int(Layout<N, KB, STAGES, HALO>::BYTES));
  return e;
}

template <int N, int KB, bool UP>
cudaError_t prepare_nk() {
  cudaError_t e = cudaSuccess;
  if constexpr (!UP && N <= 64) e = prepare_nks<N, KB, 2, false, true>();
  if constexpr (KB != 64) {
    const cudaError_t f = prepare_nks<N, KB, stages_of<N, KB>(), UP>();
    return e == cudaSuccess ? f : e;
  } else {
    for (cudaError_t f : {prepare_nks<N, KB, 2, UP>(), prepare_nks<N, KB, 3, UP>(), prepare_nks<N, KB, 4, UP>()})
      if (e == cudaSuccess) e = f;
    return e;
  }
}

// One launch: grid (pixel tiles, column blocks of N of the c.cout columns)
template <int N, int KB, int STAGES, bool UP, bool HALO = false>
cudaError_t launch_nks(const ConvTC &c, cudaStream_t s, int nblk) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  CUtensorMap ta, tb;
  // input: {channels (the buffer's channel stride), W, H, B}; box {KB, BW, BH, 1}
  const cuuint64_t adim[4] = {cuuint64_t(c.in_cs), cuuint64_t(c.W), cuuint64_t(c.H), cuuint64_t(c.B)};
  const cuuint64_t astr[3] = {cuuint64_t(c.in_cs) * 2, cuuint64_t(c.in_cs) * 2 * c.W,
                              cuuint64_t(c.in_cs) * 2 * c.W * c.H};
  const int BW = c.W >= kM ? kM : (1 << (31 - __builtin_clz(unsigned(c.W))));
  const int BH = kM / BW;
  if (HALO && BW != kM) return cudaErrorInvalidValue;
  // the halo box is one image row of the tile and one pixel on either side
  const cuuint32_t abox[4] = {cuuint32_t(KB), cuuint32_t(HALO ? kHaloPix : BW), cuuint32_t(HALO ? 1 : BH), 1};
  const cuuint32_t one[4] = {1, 1, 1, 1};
  if (fn(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16 *>(c.in), adim, astr, abox, one,
         CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_of(KB), CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  // weights [cout][9][cin]: {9 cin, cout}, or of the transposed convolution
  // [4 up_cout][cin]: {cin, 4 up_cout}; box {KB, N}
  const int taps = UP ? 1 : 9;
  const cuuint64_t bdim[2] = {cuuint64_t(taps) * c.cin, cuuint64_t(UP ? 4 * c.up_cout : c.cout)};
  const cuuint64_t bstr[1] = {cuuint64_t(taps) * c.cin * 2};
  const cuuint32_t bbox[2] = {cuuint32_t(KB), cuuint32_t(N)};
  if (fn(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16 *>(c.w), bdim, bstr, bbox, one,
         CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_of(KB), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  TCArgs a;
  a.out = c.out;
  a.out_cs = c.out_cs;
  a.out_off = c.out_off;
  a.bias = c.bias;
  a.relu = c.relu;
  a.B = c.B;
  a.H = c.H;
  a.W = c.W;
  a.cin = c.cin;
  a.in_off = c.in_off;
  a.BW = BW;
  a.BH = BH;
  a.tiles_w = (c.W + BW - 1) / BW;
  a.tiles_h = (c.H + BH - 1) / BH;
  a.n_base = c.n_base;
  a.up_cout = c.up_cout;
  a.err = c.err;
  auto k = k_conv3x3_tc<N, KB, STAGES, UP, HALO>;
  const cudaError_t e = prepare_nks<N, KB, STAGES, UP, HALO>();
  if (e != cudaSuccess) return e;
  const long long tiles = (long long)a.tiles_w * a.tiles_h * c.B;
  k<<<dim3(unsigned(tiles), unsigned(nblk)), kThreads, Layout<N, KB, STAGES, HALO>::BYTES, s>>>(ta, tb, a);
  return cudaGetLastError();
}

template <int N, int KB, bool UP>
cudaError_t launch_nk(const ConvTC &c, cudaStream_t s, int nblk, long long ctas, int sms) {
  // the halo loads for the 3x3 convolutions of up to 64 columns on images at
  // least one tile wide (32 -> 32 at 1032 x 512: 42.5 -> 34.9 us; 128 -> 64 at
  // 516 x 256: 34.3 -> 31.1 us); with 128 columns it was slower
  if constexpr (!UP && N <= 64)
    if (c.W >= kM) return launch_nks<N, KB, 2, false, true>(c, s, nblk);
  if constexpr (KB != 64) {
    return launch_nks<N, KB, stages_of<N, KB>(), UP>(c, s, nblk);
  } else {
    if (ctas <= (long long)sms * occupancy_of<N, KB, 4>()) return launch_nks<N, KB, 4, UP>(c, s, nblk);
    if (ctas <= (long long)sms * occupancy_of<N, KB, 3>()) return launch_nks<N, KB, 3, UP>(c, s, nblk);
    return launch_nks<N, KB, 2, UP>(c, s, nblk);
  }
}

template <int N, bool UP>
cudaError_t launch_n(const ConvTC &c, cudaStream_t s, int nblk, long long ctas, int sms) {
  if (c.cin % 64 == 0) return launch_nk<N, 64, UP>(c, s, nblk, ctas, sms);
  if (c.cin % 32 == 0) return launch_nk<N, 32, UP>(c, s, nblk, ctas, sms);
  return launch_nk<N, 16, UP>(c, s, nblk, ctas, sms);
}

constexpr int kUpbStages = 3;
template <int N, int KB>
cudaError_t prepare_upb() {
  static cudaError_t e = cudaFuncSetAttribute(k_conv3x3_tc<N, KB, kUpbStages, false, false, true>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              int(Layout<N, KB, kUpbStages>::BYTES));
  return e;
}

template <int N>
cudaError_t prepare_n() {
  cudaError_t e = cudaSuccess;
  for (cudaError_t f : {prepare_nk<N, 64, false>(), prepare_nk<N, 32, false>(), prepare_nk<N, 16, false>(),
                        prepare_nk<N, 64, true>(), prepare_nk<N, 32, true>(), prepare_nk<N, 16, true>(),
                        prepare_upb<N, 64>(), prepare_upb<N, 32>(), prepare_upb<N, 16>()})
    if (e == cudaSuccess) e = f;
  return e;
}

// Data gradient of the transposed convolution (UPB): grid (pixel tiles of
// the transposed convolution's input, column blocks of its input channels)
template <int N, int KB>
cudaError_t launch_upb(const ConvTC &c, cudaStream_t s, int nblk) {
  constexpr int STAGES = kUpbStages;
  using L = Layout<N, KB, STAGES>;
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cudaError_t attr = prepare_upb<N, KB>();
  if (attr != cudaSuccess) return attr;
  CUtensorMap ta, tb;
  // the output gradient [B][2H][2W][in_cs] as {channels, c, x, a, B H}: child (a, c)
  // of input pixel (y, x) is (2y + a, 2x + c)
  const cuuint64_t e = 2;   // bytes per element
  const cuuint64_t adim[5] = {cuuint64_t(c.in_cs), 2, cuuint64_t(c.W), 2, cuuint64_t(c.B) * c.H};
  const cuuint64_t astr[4] = {cuuint64_t(c.in_cs) * e, cuuint64_t(c.in_cs) * e * 2,
                              cuuint64_t(c.in_cs) * e * 2 * c.W, cuuint64_t(c.in_cs) * e * 4 * c.W};
  const int BW = c.W >= kM ? kM : (1 << (31 - __builtin_clz(unsigned(c.W))));
  const int BH = kM / BW;
  const cuuint32_t abox[5] = {cuuint32_t(KB), 1, cuuint32_t(BW), 1, cuuint32_t(BH)};
  const cuuint32_t one[5] = {1, 1, 1, 1, 1};
  if (fn(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16 *>(c.in), adim, astr, abox, one,
         CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_of(KB), CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  // weights [4 ncols][K]: {K, 4 ncols}; box {KB, N}
  const cuuint64_t bdim[2] = {cuuint64_t(c.cin), cuuint64_t(4) * c.cout};
  const cuuint64_t bstr[1] = {cuuint64_t(c.cin) * e};
  const cuuint32_t bbox[2] = {cuuint32_t(KB), cuuint32_t(N)};
  if (fn(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16 *>(c.w), bdim, bstr, bbox, one,
         CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_of(KB), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  TCArgs a;
  a.out = c.out;
  a.out_cs = c.out_cs;
  a.out_off = c.out_off;
  a.bias = nullptr;
  a.relu = 0;
  a.B = c.B;
  a.H = c.H;
  a.W = c.W;
  a.cin = c.cin;
  a.in_off = c.in_off;
  a.BW = BW;
  a.BH = BH;
  a.tiles_w = (c.W + BW - 1) / BW;
  a.tiles_h = (c.H + BH - 1) / BH;
  a.n_base = 0;
  a.up_cout = 0;
  a.ncols = c.cout;
  a.err = c.err;
  const long long tiles = (long long)a.tiles_w * a.tiles_h * c.B;
  k_conv3x3_tc<N, KB, STAGES, false, false, true>
      <<<dim3(unsigned(tiles), unsigned(nblk)), kThreads, L::BYTES, s>>>(ta, tb, a);
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_upb_n(const ConvTC &c, cudaStream_t s, int nblk) {
  if (c.cin % 64 == 0) return launch_upb<N, 64>(c, s, nblk);
  if (c.cin % 32 == 0) return launch_upb<N, 32>(c, s, nblk);
  return launch_upb<N, 16>(c, s, nblk);
}

constexpr int kWStages = 3;
template <int CO, int CI, bool UPW = false>
cudaError_t prepare_wgrad() {
  static cudaError_t e = cudaFuncSetAttribute(k_wgrad_tc<CO, CI, kWStages, UPW>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              int(WLayout<CO, CI, kWStages, UPW>::BYTES));
  return e;
}

// CTAs of one wave over yb (co, ci) blocks, each a run of K blocks (at least one)
template <class L>
long long wgrad_split(WArgs &a, int sms, int yb) {
  const int res_smem = int((227u * 1024u) / L::BYTES), res_tmem = int(512u / L::NCOLS);
  const int res = res_smem < res_tmem ? (res_smem > 0 ? res_smem : 1) : res_tmem;
  long long splits = ((long long)sms * res + yb - 1) / yb;
  if (splits > a.nkb) splits = a.nkb;
  if (splits < 1) splits = 1;
  a.per_cta = (a.nkb + splits - 1) / splits;
  return (a.nkb + a.per_cta - 1) / a.per_cta;
}

template <int CO, int CI>
cudaError_t launch_wgrad(const WgradTC &g, cudaStream_t s, int sms) {
  using L = WLayout<CO, CI, kWStages>;
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cudaError_t attr = prepare_wgrad<CO, CI>();
  if (attr != cudaSuccess) return attr;
  const cuuint64_t e = 2;
  const cuuint32_t one[4] = {1, 1, 1, 1};
  CUtensorMap ta, tb;
  // the gradient [B][H][W][cout] as {cout, W, H, B}, boxes {CO, 64 pixels}
  const cuuint64_t adim[4] = {cuuint64_t(g.cout), cuuint64_t(g.W), cuuint64_t(g.H), cuuint64_t(g.B)};
  const cuuint64_t astr[3] = {cuuint64_t(g.cout) * e, cuuint64_t(g.cout) * e * g.W, cuuint64_t(g.cout) * e * g.W * g.H};
  const cuuint32_t abox[4] = {cuuint32_t(CO), cuuint32_t(kWKP), 1, 1};
  if (fn(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16 *>(g.dpre), adim, astr, abox, one,
         CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_of(CO), CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  // the input [B][H][W][in_cs] as {in_cs, W, H, B}, boxes {CI, 80 pixels}
  const cuuint64_t bdim[4] = {cuuint64_t(g.in_cs), cuuint64_t(g.W), cuuint64_t(g.H), cuuint64_t(g.B)};
  const cuuint64_t bstr[3] = {cuuint64_t(g.in_cs) * e, cuuint64_t(g.in_cs) * e * g.W,
                              cuuint64_t(g.in_cs) * e * g.W * g.H};
  const cuuint32_t bbox[4] = {cuuint32_t(CI), cuuint32_t(L::KPB), 1, 1};
  if (fn(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16 *>(g.in), bdim, bstr, bbox, one,
         CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_of(CI), CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  WArgs a;
  a.dw = g.dw;
  a.cin = g.cin;
  a.cout = g.cout;
  a.in_off = g.in_off;
  a.a_off = 0;
  a.H = g.H;
  a.nwc = (g.W + kWKP - 1) / kWKP;
  a.nkb = (long long)g.B * g.H * a.nwc;
  a.err = g.err;
  // one wave: the CTAs that fit on the SMs at once (shared memory, TMEM
  // columns), shared out over the (co, ci) blocks, each a run of K blocks
  const int yb = (g.cout / CO) * (g.cin / CI);
  const long long splits = wgrad_split<L>(a, sms, yb);
  k_wgrad_tc<CO, CI, kWStages><<<dim3(unsigned(splits), unsigned(yb)), kThreads, L::BYTES, s>>>(ta, tb, a);
  return cudaGetLastError();
}

template <int CO>
cudaError_t launch_upw(const UpWgradTC &g, cudaStream_t s, int sms) {
  constexpr int CI = 64;
  using L = WLayout<CO, CI, kWStages, true>;
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cudaError_t attr = prepare_wgrad<CO, CI, true>();
  if (attr != cudaSuccess) return attr;
  const cuuint64_t e = 2;
  const cuuint32_t one[5] = {1, 1, 1, 1, 1};
  CUtensorMap ta, tb;
  // the output gradient [B][2H][2W][g_cs] as {g_cs, c, x, a, B H}: child (a, c)
  // of input pixel (y, x) is (2y + a, 2x + c); boxes {CO, 1, 64, 1, 1}
  const cuuint64_t adim[5] = {cuuint64_t(g.g_cs), 2, cuuint64_t(g.W), 2, cuuint64_t(g.B) * g.H};
  const cuuint64_t astr[4] = {cuuint64_t(g.g_cs) * e, cuuint64_t(g.g_cs) * e * 2, cuuint64_t(g.g_cs) * e * 2 * g.W,
                              cuuint64_t(g.g_cs) * e * 4 * g.W};
  const cuuint32_t abox[5] = {cuuint32_t(CO), 1, cuuint32_t(kWKP), 1, 1};
  if (fn(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16 *>(g.g), adim, astr, abox, one,
         CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_of(CO), CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  // the input [B][H][W][cin] as {cin, W, H, B}, boxes {64, 80 pixels} from 8 before
  const cuuint64_t bdim[4] = {cuuint64_t(g.cin), cuuint64_t(g.W), cuuint64_t(g.H), cuuint64_t(g.B)};
  const cuuint64_t bstr[3] = {cuuint64_t(g.cin) * e, cuuint64_t(g.cin) * e * g.W, cuuint64_t(g.cin) * e * g.W * g.H};
  const cuuint32_t bbox[4] = {cuuint32_t(CI), cuuint32_t(L::KPB), 1, 1};
  if (fn(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16 *>(g.in), bdim, bstr, bbox, one,
         CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_of(CI), CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  WArgs a;
  a.dw = g.dw;
  a.cin = g.cin;
  a.cout = g.cout;
  a.in_off = 0;
  a.a_off = g.g_off;
  a.H = g.H;
  a.nwc = (g.W + kWKP - 1) / kWKP;
  a.nkb = (long long)g.B * g.H * a.nwc;
  a.err = g.err;
  const int yb = (g.cout / CO) * (g.cin / CI);
  const long long splits = wgrad_split<L>(a, sms, yb);
  k_wgrad_tc<CO, CI, kWStages, true><<<dim3(unsigned(splits), unsigned(yb)), kThreads, L::BYTES, s>>>(ta, tb, a);
  return cudaGetLastError();
}

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return sms;
}

}  // namespace tc

cudaError_t conv3x3_tc_prepare() {
  cudaError_t e = tc::prepare_n<32>();
  if (e == cudaSuccess) e = tc::prepare_n<64>();
  if (e == cudaSuccess) e = tc::prepare_n<128>();
  if (e == cudaSuccess) e = tc::prepare_n<256>();
  for (cudaError_t f : {tc::prepare_wgrad<32, 16>(), tc::prepare_wgrad<32, 32>(), tc::prepare_wgrad<32, 64>(),
                        tc::prepare_wgrad<64, 16>(), tc::prepare_wgrad<64, 32>(), tc::prepare_wgrad<64, 64>(),
                        tc::prepare_wgrad<32, 64, true>(), tc::prepare_wgrad<64, 64, true>()})
    if (e == cudaSuccess) e = f;
  return e;
}

bool conv3x3_tc_supported(int cin, int cout, int in_cs, int in_off, int out_cs, int out_off, int W) {
  return cin >= 16 && cin % 16 == 0 && (cout == 32 || cout == 64 || cout == 128 || cout == 256) &&
         in_cs % 8 == 0 && in_off % 8 == 0 && out_cs % 8 == 0 && out_off % 8 == 0 && W >= 8 &&
         tc::encode_fn() != nullptr;
}

cudaError_t conv3x3_tc(const ConvTC &c, cudaStream_t s) {
  if (!conv3x3_tc_supported(c.cin, c.cout, c.in_cs, c.in_off, c.out_cs, c.out_off, c.W))
    return cudaErrorNotSupported;
  // the transposed convolution's GEMM columns come in launches of at most 256
  if (c.up_cout && (c.up_cout % 16 || c.n_base % c.up_cout || c.n_base + c.cout > 4 * c.up_cout))
    return cudaErrorNotSupported;
  const int sms = tc::sm_count();
  if (sms < 1) return cudaErrorInvalidValue;
  const int BW = c.W >= tc::kM ? tc::kM : (1 << (31 - __builtin_clz(unsigned(c.W))));
  const long long tiles = (long long)((c.W + BW - 1) / BW) * ((c.H + tc::kM / BW - 1) / (tc::kM / BW)) * c.B;
  // column blocks while the pixel tiles alone leave SMs idle
  int n = c.cout, nblk = 1;
  while (n > 64 && tiles * nblk < sms) {
    n >>= 1;
    nblk <<= 1;
  }
  const long long ctas = tiles * nblk;
  const bool up = c.up_cout != 0;
  switch (n) {
    case 32: return up ? tc::launch_n<32, true>(c, s, nblk, ctas, sms) : tc::launch_n<32, false>(c, s, nblk, ctas, sms);
    case 64: return up ? tc::launch_n<64, true>(c, s, nblk, ctas, sms) : tc::launch_n<64, false>(c, s, nblk, ctas, sms);
    case 128: return up ? tc::launch_n<128, true>(c, s, nblk, ctas, sms) : tc::launch_n<128, false>(c, s, nblk, ctas, sms);
    default: return up ? tc::launch_n<256, true>(c, s, nblk, ctas, sms) : tc::launch_n<256, false>(c, s, nblk, ctas, sms);
  }
}

cudaError_t conv_in_tc(const float2 *x, const __nv_bfloat16 *w, int wcin, const float *bias,
                       __nv_bfloat16 *out, int B, int H, int W, int relu, int *err, cudaStream_t s) {
  const int sms = tc::sm_count();
  if (sms < 1 || wcin < tc::kInCh) return cudaErrorInvalidValue;
  const long long npix = (long long)B * H * W;
  if (npix < 1 || npix >= (1LL << 31)) return cudaErrorInvalidValue;
  const long long ntiles = (npix + tc::kM - 1) / tc::kM;
  const long long grid = ntiles < 8LL * sms ? ntiles : 8LL * sms;   // 8 CTAs per SM, tiles in turn
  tc::k_conv_in_tc<<<unsigned(grid), tc::kThreads, 0, s>>>(x, w, wcin, bias, out, B, H, W, relu, err);
  return cudaGetLastError();
}

cudaError_t conv_upback_tc(const ConvTC &c, cudaStream_t s) {
  if (!conv3x3_tc_supported(c.cin, c.cout, c.in_cs, c.in_off, c.out_cs, c.out_off, c.W) ||
      (long long)c.B * c.H >= (1LL << 31))
    return cudaErrorNotSupported;
  const int sms = tc::sm_count();
  if (sms < 1) return cudaErrorInvalidValue;
  const int BW = c.W >= tc::kM ? tc::kM : (1 << (31 - __builtin_clz(unsigned(c.W))));
  const long long tiles = (long long)((c.W + BW - 1) / BW) * ((c.H + tc::kM / BW - 1) / (tc::kM / BW)) * c.B;
  int n = c.cout, nblk = 1;
  while (n > 64 && tiles * nblk < sms) {
    n >>= 1;
    nblk <<= 1;
  }
  switch (n) {
    case 32: return tc::launch_upb_n<32>(c, s, nblk);
    case 64: return tc::launch_upb_n<64>(c, s, nblk);
    case 128: return tc::launch_upb_n<128>(c, s, nblk);
    default: return tc::launch_upb_n<256>(c, s, nblk);
  }
}

bool conv_wgrad_tc_supported(int cin, int cout, int in_cs, int in_off, const float *dw) {
  return (cout == 32 || (cout >= 64 && cout % 64 == 0)) && (cin == 16 || cin == 32 || (cin >= 64 && cin % 64 == 0)) &&
         in_cs % 8 == 0 && in_off % 8 == 0 && in_off + cin <= in_cs && (reinterpret_cast<uintptr_t>(dw) & 15) == 0 &&
         tc::encode_fn() != nullptr;
}

cudaError_t conv_wgrad_tc(const WgradTC &g, cudaStream_t s) {
  if (!conv_wgrad_tc_supported(g.cin, g.cout, g.in_cs, g.in_off, g.dw) || g.B < 1 || g.H < 1 || g.W < 1)
    return cudaErrorNotSupported;
  const int sms = tc::sm_count();
  if (sms < 1) return cudaErrorInvalidValue;
  const int ci = g.cin >= 64 ? 64 : g.cin;
  if (g.cout == 32) {
    if (ci == 16) return tc::launch_wgrad<32, 16>(g, s, sms);
    if (ci == 32) return tc::launch_wgrad<32, 32>(g, s, sms);
    return tc::launch_wgrad<32, 64>(g, s, sms);
  }
  if (ci == 16) return tc::launch_wgrad<64, 16>(g, s, sms);
  if (ci == 32) return tc::launch_wgrad<64, 32>(g, s, sms);
  return tc::launch_wgrad<64, 64>(g, s, sms);
}

bool conv_upwgrad_tc_supported(int cin, int cout, int g_cs, int g_off) {
  return (cout == 32 || (cout >= 64 && cout % 64 == 0)) && cin >= 64 && cin % 64 == 0 && g_cs % 8 == 0 &&
         g_off % 8 == 0 && g_off + cout <= g_cs && tc::encode_fn() != nullptr;
}

cudaError_t conv_upwgrad_tc(const UpWgradTC &g, cudaStream_t s) {
  if (!conv_upwgrad_tc_supported(g.cin, g.cout, g.g_cs, g.g_off) || g.B < 1 || g.H < 1 || g.W < 1 ||
      (long long)g.B * g.H >= (1LL << 31))
    return cudaErrorNotSupported;
  const int sms = tc::sm_count();
  if (sms < 1) return cudaErrorInvalidValue;
  return g.cout == 32 ? tc::launch_upw<32>(g, s, sms) : tc::launch_upw<64>(g, s, sms);
}

}  // namespace picgb
