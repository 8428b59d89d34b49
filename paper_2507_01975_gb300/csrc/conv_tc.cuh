// conv_tc.cuh -- 3x3 periodic convolutions of the learnable module on the
// 5th-generation tensor cores (tcgen05, BF16 in, FP32 accumulate in TMEM).
//
// The stencil network C_theta (6 conv3x3 layers, GELU between them) and the
// temporal-correction network run at every RK stage; their hidden layers
// (64 -> 64 and 64 -> 160 channels) are implicit GEMMs:
//   out[p][co] = b[co] + sum_{dy,dx,ci} W[co][ci][dy][dx] in[p + (dy,dx)][ci].
//
// Activation layout in global memory ("chunk planes"): [batch][C/8][N][N][8]
// BF16, i.e. for each group of 8 channels one N x N plane of 16-byte pixels.
// A tile of 128 output pixels (128/N image rows) needs input rows y0-1 ..
// y0+128/N; in shared memory each 8-channel plane of those rows is contiguous,
// which is exactly the no-swizzle K-major operand layout of tcgen05.mma
// (8-pixel x 16-byte core matrices, M-stride 128 B, K-stride one plane). A
// shift by dy is a start-address offset of one image row. Shifts by dx would
// wrap around the row ends (periodic padding), so instead the three dx
// columns of the kernel accumulate into three TMEM accumulators P_dx over the
// *unshifted* pixels -- one MMA with N = 3 x COUT_TILE (the weights of the
// three dx taps side by side) produces all three -- and the epilogue forms
// out[x] = P_-1[x-1] + P_0[x] + P_+1[x+1] with the periodic wrap.
//
// Roles (20 warps): warp 0 lane 0 issues the bulk copies of the input tiles
// (double buffered, mbarrier transaction counts), warp 1 allocates TMEM and
// its lane 0 issues the MMAs, warps 4..19 run the epilogue (four warps per
// TMEM lane quarter, each taking a quarter of the output channels). Accumulators are
// double buffered so the epilogue of one tile overlaps the MMAs of the next.
// Every mbarrier wait is bounded; on time-out the CTA records an error and
// stops issuing work.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "fv_common.cuh"

namespace ldfv {

struct ConvArgs {
  const __nv_bfloat16* in;   // [batch][CIN/8][N][N][8]
  const __nv_bfloat16* w;    // packed: [parts][9 taps][CIN/8][COUT_TILE/8][8 co][8 ci]
  const float* bias;         // [COUT_TOTAL]
  __nv_bfloat16* out;        // [batch][COUT_TOTAL/8][N][N][8]
  int batch;
  int parts;                 // output-channel parts of COUT_TILE channels each
  int co_base;               // first output channel of part 0
  int cout_total;            // channel count of the output tensor
  int gelu;                  // epilogue: 0 none, 1 GELU (pre-activation to aux if set),
                             // 2 multiply by GELU'(aux) (reverse mode of GELU, no bias)
  const __nv_bfloat16* aux_in;  // mode 2: pre-activation, same layout as out
  __nv_bfloat16* aux_out;       // mode 1: pre-activation is stored here when non-null
  unsigned* err;             // set to nonzero on a timed-out wait
  long long spin_limit;
  float* dbias;              // mode 2: per-channel sums of the FP32 output added here (atomics), or null
};

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05; no swizzle, base offset 0
  return d;
}

// kind::f16 instruction descriptor: BF16 A and B, FP32 D, both K-major
template <int M, int N>
__host__ __device__ constexpr uint32_t umma_idesc_bf16() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
// bounded wait for completion of the phase with parity `par`; false on time-out
// Iteration limit of the waits that drain a CTA's own asynchronous work
// (bulk copies, MMAs) before it exits after an error: independent of the
// caller's limit, which can be small enough to make the regular waits give up.
constexpr long long kDrainSpin = 1ll << 20;

__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t par, long long limit) {
  for (long long it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(par)
        : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void umma_bf16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void tmem_ld8f(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  tmem_ld8(taddr, r);
  tmem_wait_ld();
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

// 16 or 32 consecutive FP32 columns of this thread's TMEM lane; the caller
// issues tmem_wait_ld() before using the values
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, float (&v)[16]) {
  uint32_t* r = reinterpret_cast<uint32_t*>(v);
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, float* v) {
  uint32_t* r = reinterpret_cast<uint32_t*>(v);
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}
template <int NC>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, float (&v)[NC]) {
  static_assert(NC % 8 == 0, "8-column loads");
  if constexpr (NC % 16 == 0) {
#pragma unroll
    for (int k = 0; k < NC / 16; ++k) tmem_ld16_nowait(taddr + 16 * k, *reinterpret_cast<float(*)[16]>(v + 16 * k));
  } else {
#pragma unroll
    for (int k = 0; k < NC / 8; ++k) tmem_ld8_nowait(taddr + 8 * k, v + 8 * k);
  }
}

// GELU(x) = x Phi(x) = 0.5 x (1 + erf(x / sqrt 2)) of the forward epilogues,
// with erf(z) ~ tanh(z (a + b z^2)): a = 1.12967583, b = 0.0997927 minimise the
// largest error over z >= 0 (2.8e-4; fitted here), so
// GELU(x) ~ 0.5 x (1 + tanh(x (A + B x^2))), A = a / sqrt 2, B = b / (2 sqrt 2),
// evaluated with the hardware tanh (one special-function op per value; its
// relative error is 2^-11). The result is within 4e-4 + 2.5e-4 |x| of GELU,
// below the BF16 rounding of the activations it produces (2^-9 relative).
__device__ __forceinline__ float tanh_hw(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float gelu_f(float x) {
  const float y = x * fmaf(0.0352820483f, x * x, 0.798801437f);
  const float h = 0.5f * x;
  return fmaf(h, tanh_hw(y), h);
}

// Packed FP32 pairs: one add / mul / fma instruction for two values (the
// epilogue's arithmetic is elementwise, so its values go in pairs).
struct f32x2 {
  unsigned long long v;
};
__device__ __forceinline__ f32x2 pack2(float a, float b) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void unpack2(f32x2 p, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(p.v));
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}
// gelu_f on a pair
__device__ __forceinline__ f32x2 gelu2(f32x2 x) {
  const f32x2 y = mul2(x, fma2(mul2(x, x), pack2(0.0352820483f, 0.0352820483f), pack2(0.798801437f, 0.798801437f)));
  const f32x2 h = mul2(x, pack2(0.5f, 0.5f));
  float y0, y1;
  unpack2(y, y0, y1);
  return fma2(h, pack2(tanh_hw(y0), tanh_hw(y1)), h);
}

// The same GELU with erf from the rational approximation 7.1.26 of Abramowitz &
// Stegun (|error| <= 1.5e-7): the reference form of the derivative below.

// GELU'(x) = Phi(x) + x phi(x), with the same erf approximation
__device__ __forceinline__ float gelu_grad_f(float x) {
  const float z = fabsf(x) * 0.70710678118654752f;
  const float t = __fdividef(1.0f, 1.0f + 0.3275911f * z);
  const float poly = t * (0.254829592f + t * (-0.284496736f + t * (1.421413741f + t * (-1.453152027f + t * 1.061405429f))));
  const float g = __expf(-z * z);
  const float erf_abs = 1.0f - poly * g;
  const float erf_x = x < 0.0f ? -erf_abs : erf_abs;
  return 0.5f * (1.0f + erf_x) + x * 0.39894228040143268f * g;
}

template <int LOGN, int CIN, int COUT_TILE, int NBUF = (LOGN >= 7 ? 3 : 4)>
struct ConvCfg {
  static constexpr int N = 1 << LOGN;
  static constexpr int TM = 128;             // output pixels per tile
  static constexpr int TROWS = TM / N;       // image rows per tile
  static constexpr int IROWS = TROWS + 2;    // input rows with the dy halo
  static constexpr int KC = CIN / 8;         // 8-channel chunks
  // epilogue warps: 4 per TMEM lane quarter; warps 0 .. 3 are the producer,
  // the MMA issuer and two idle warps (640 threads; more epilogue warps would
  // pass the 1024-thread limit of a CTA)
  static constexpr int NEPI = 16;
  static constexpr int NT = 128 + NEPI * 32;
  static constexpr int CG = COUT_TILE * 4 / NEPI;  // output channels per epilogue warp
  static constexpr uint32_t PLANE_BYTES = IROWS * N * 16;         // one chunk plane of the tile
  static constexpr uint32_t ATILE_BYTES = KC * PLANE_BYTES;       // one input tile
  // weights [dy][c8][dx][co8][8 co][8 ci]: the three dx blocks of one (dy, c8)
  // are adjacent along N, so one MMA with N = 3 COUT_TILE produces P_-1, P_0, P_+1
  static constexpr uint32_t KSTEP_BYTES = 3 * (COUT_TILE / 8) * 128;  // one c8 of one dy
  static constexpr uint32_t W_BYTES = 3 * KC * KSTEP_BYTES;
  static constexpr uint32_t OFF_A = 0;                            // NBUF input tiles
  static constexpr uint32_t OFF_W = NBUF * ATILE_BYTES;
  static constexpr uint32_t OFF_BND = OFF_W + W_BYTES;            // epilogue boundary exchange
  static constexpr uint32_t BND_BYTES = 2 * (NEPI / 4) * 4 * 2 * CG * 4;  // [parity][group][quarter][2][CG]
  static constexpr uint32_t OFF_BIASV = OFF_BND + BND_BYTES;      // bias of the whole output tensor
  static constexpr uint32_t OFF_BAR = OFF_BIASV + 256 * 4;
  static constexpr uint32_t OFF_PAIR = OFF_BAR + 128;             // per exchange-group abort flags
  static constexpr uint32_t SMEM = OFF_PAIR + 64;
  // epilogue warps of one channel group that hold the lane quarters of one
  // image row exchange edge values: QR quarters per row, groups of QR warps
  // (none for N = 32, where a quarter is a whole row)
  static constexpr int QR = N / 32;
  static constexpr int NXG = QR > 1 ? (NEPI / 4) * (4 / QR) : 0;  // exchange groups
  static_assert(NXG <= 8, "named barriers 2 .. 9; abort flags [tile parity][group]");
  static constexpr int ACC_COLS = 3 * COUT_TILE;                  // P_-1, P_0, P_+1
  static constexpr int TMEM_COLS = 2 * ACC_COLS <= 256 ? 256 : 512;
  static_assert(N >= 32 && N <= 128, "a tile covers whole image rows");
  static_assert(CIN % 16 == 0, "K steps of 16");
  static_assert(COUT_TILE % 32 == 0 && COUT_TILE >= 32 && 3 * COUT_TILE <= 256, "accumulator width (MMA N)");
  static_assert(2 * ACC_COLS <= 512, "double-buffered accumulators fit tensor memory");
  static_assert(SMEM <= 232448, "shared memory");
  static_assert(PLANE_BYTES < (1u << 18), "descriptor offsets");
  static_assert(NBUF >= 1 && NBUF <= 4, "input buffering");
};

template <int LOGN, int CIN, int COUT_TILE, int NBUF = (LOGN >= 7 ? 3 : 4)>
__global__ void __launch_bounds__(ConvCfg<LOGN, CIN, COUT_TILE, NBUF>::NT, 1) conv3x3_tc_kernel(const ConvArgs a) {
  using Cfg = ConvCfg<LOGN, CIN, COUT_TILE, NBUF>;
  constexpr int N = Cfg::N, TROWS = Cfg::TROWS, IROWS = Cfg::IROWS, KC = Cfg::KC;
  constexpr int CG = Cfg::CG;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* const sA = smem + Cfg::OFF_A;
  unsigned char* const sW = smem + Cfg::OFF_W;
  float* const bnd = reinterpret_cast<float*>(smem + Cfg::OFF_BND);
  float* const sbias = reinterpret_cast<float*>(smem + Cfg::OFF_BIASV);
  uint64_t* const bars = reinterpret_cast<uint64_t*>(smem + Cfg::OFF_BAR);
  uint64_t* const a_full = bars + 0;    // [NBUF] input tile landed
  uint64_t* const a_empty = bars + 4;   // [NBUF] MMAs of the input tile done
  uint64_t* const c_full = bars + 8;    // [2] accumulator ready
  uint64_t* const c_empty = bars + 10;  // [2] accumulator read out
  uint64_t* const w_full = bars + 12;
  uint32_t* const tslot = reinterpret_cast<uint32_t*>(bars + 13);
  volatile uint32_t* const abort_flag = reinterpret_cast<volatile uint32_t*>(bars + 14);
  volatile uint32_t* const pair_abort = reinterpret_cast<volatile uint32_t*>(smem + Cfg::OFF_PAIR);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tiles_per_img = N / TROWS;
  const int npix = a.batch * tiles_per_img;  // pixel tiles per part
  const int ntiles = npix * a.parts;         // part-major: a CTA rarely changes part
  const long long lim = a.spin_limit;

  if (tid == 0) {
    for (int s = 0; s < NBUF; ++s) {
      mbar_init(a_full + s, 1);
      mbar_init(a_empty + s, 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(c_full + s, 1);
      mbar_init(c_empty + s, Cfg::NEPI * 32);
    }
    mbar_init(w_full, 1);
    *abort_flag = 0;
    for (int g = 0; g < 16; ++g) pair_abort[g] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tslot, Cfg::TMEM_COLS);
  for (int k = tid; k < a.cout_total; k += Cfg::NT) sbias[k] = a.bias ? a.bias[k] : 0.0f;
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tmem = *tslot;
  // the first part's weights were written two or more launches back (every
  // kernel here waits for its predecessor before it lets its successor
  // launch), so their copy starts before the wait, overlapping the previous
  // kernel's tail
  const int first_part = (int)blockIdx.x < ntiles ? (int)blockIdx.x / npix : -1;
  if (warp == 0 && lane == 0 && first_part >= 0) {
    mbar_expect_tx(w_full, Cfg::W_BYTES);
    const unsigned char* wsrc = reinterpret_cast<const unsigned char*>(a.w) + (size_t)first_part * Cfg::W_BYTES;
    for (uint32_t off = 0; off < Cfg::W_BYTES; off += 16384) {
      const uint32_t sz = (Cfg::W_BYTES - off) < 16384 ? (Cfg::W_BYTES - off) : 16384;
      bulk_g2s(sW + off, wsrc + off, sz, w_full);
    }
  }
  // the rest of the prologue overlaps the previous kernel's tail; the inputs
  // and the outputs' previous readers belong to the previous kernel
  pdl_wait();
  pdl_trigger();

  if (warp == 0) {
    // ---------------- producer: weights once per part change, input tiles ----------
    // lane 0 waits and arms the barriers; all 32 lanes issue the tile's copies
    int cur_part = first_part;
    uint32_t wphase_waits = first_part >= 0 ? 1u : 0u;
    int i = 0;
    int issued = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int part = t / npix;
      const int pix = t % npix;
      const int b = pix / tiles_per_img, y0 = (pix % tiles_per_img) * TROWS;
      const int s = i % NBUF;
      const uint32_t aph = (uint32_t)((i / NBUF) & 1);
      int ok = 1;
      if (lane == 0) {
        if (!mbar_wait(a_empty + s, aph ^ 1, lim)) {
          ok = 0;
          atomicOr(a.err, 1u);
        } else if (part != cur_part) {
          // the MMAs of every earlier tile have completed once the previous
          // tile's commit has arrived (commits track all prior MMAs), so the
          // weight area can be overwritten
          if (i > 0 && !mbar_wait(a_empty + (i - 1) % NBUF, (uint32_t)(((i - 1) / NBUF) & 1), lim)) {
            ok = 0;
            atomicOr(a.err, 2u);
          } else {
            mbar_expect_tx(w_full, Cfg::W_BYTES);
            const unsigned char* wsrc = reinterpret_cast<const unsigned char*>(a.w) + (size_t)part * Cfg::W_BYTES;
            for (uint32_t off = 0; off < Cfg::W_BYTES; off += 16384) {
              const uint32_t sz = (Cfg::W_BYTES - off) < 16384 ? (Cfg::W_BYTES - off) : 16384;
              bulk_g2s(sW + off, wsrc + off, sz, w_full);
            }
          }
        }
        if (ok) mbar_expect_tx(a_full + s, Cfg::ATILE_BYTES);
        if (!ok) *abort_flag = 1;
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      if (part != cur_part) {
        cur_part = part;
        ++wphase_waits;
      }
      __syncwarp();
      // rows y0 - 1 .. y0 + TROWS of each plane are contiguous in global memory
      // except across the periodic wrap: one copy per plane, two at the wrap
      unsigned char* dst = sA + s * Cfg::ATILE_BYTES;
      for (int c = lane; c < KC; c += 32) {
        const unsigned char* plane = reinterpret_cast<const unsigned char*>(a.in + ((size_t)b * KC + c) * N * N * 8);
        unsigned char* d = dst + c * Cfg::PLANE_BYTES;
        constexpr uint32_t ROWB = N * 16;
        if (y0 == 0) {  // row -1 is row N - 1
          bulk_g2s(d, plane + (size_t)(N - 1) * ROWB, ROWB, a_full + s);
          bulk_g2s(d + ROWB, plane, (IROWS - 1) * ROWB, a_full + s);
        } else if (y0 + TROWS == N) {  // row N is row 0
          bulk_g2s(d, plane + (size_t)(y0 - 1) * ROWB, (IROWS - 1) * ROWB, a_full + s);
          bulk_g2s(d + (IROWS - 1) * ROWB, plane, ROWB, a_full + s);
        } else {
          bulk_g2s(d, plane + (size_t)(y0 - 1) * ROWB, IROWS * ROWB, a_full + s);
        }
      }
      issued = i + 1;
    }
    // never leave with bulk copies in flight: wait (bounded) for the last
    // NBUF tiles and the last weight load to land
    if (lane == 0) {
      for (int j = issued - NBUF; j < issued; ++j)
        if (j >= 0) mbar_wait(a_full + j % NBUF, (uint32_t)((j / NBUF) & 1), kDrainSpin);
      if (wphase_waits > 0) mbar_wait(w_full, (wphase_waits - 1) & 1, kDrainSpin);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer -------------------------------------------------
    if (lane == 0) {
      constexpr uint32_t idesc = umma_idesc_bf16<128, 3 * COUT_TILE>();
      int cur_part = -1;
      uint32_t wpar = 0;
      int i = 0;
      int last = -1;  // last tile whose MMAs were committed
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
        const int part = t / npix;
        const int s = i & 1;                              // accumulator buffer
        const int sa = i % NBUF;                          // input buffer
        const uint32_t aph = (uint32_t)((i / NBUF) & 1);
        if (*abort_flag) break;
        if (part != cur_part) {
          if (!mbar_wait(w_full, wpar, lim)) {
            *abort_flag = 1;
            atomicOr(a.err, 4u);
            break;
          }
          wpar ^= 1;
          cur_part = part;
        }
        if (!mbar_wait(a_full + sa, aph, lim) || !mbar_wait(c_empty + s, ((i >> 1) & 1) ^ 1, lim)) {
          *abort_flag = 1;
          atomicOr(a.err, 8u);
          break;
        }
        tmem_fence_after_sync();
        const uint32_t abase = smem_u32(sA + sa * Cfg::ATILE_BYTES);
        const uint32_t wbase = smem_u32(sW);
        const uint32_t dbase = tmem + (uint32_t)(s * Cfg::ACC_COLS);
        // descriptors of the tile's first A and B core matrices; the start
        // address field is linear (16-byte units, no carry out of it inside
        // shared memory), so every MMA's operands are these plus a constant.
        // One MMA per (dy, 16 input channels) with N = 3 COUT_TILE writes the
        // three dx accumulators at once (columns dx * COUT_TILE + co).
        const uint64_t ad0 = umma_desc(abase, Cfg::PLANE_BYTES, 128);
        const uint64_t bd0 = umma_desc(wbase, Cfg::KSTEP_BYTES, 128);
#pragma unroll
        for (int dyi = 0; dyi < 3; ++dyi) {  // dy = dyi - 1: a start offset of one image row
#pragma unroll
          for (int kk = 0; kk < KC / 2; ++kk) {
            const uint64_t ad = ad0 + (uint64_t)(((2 * kk) * Cfg::PLANE_BYTES + dyi * N * 16) >> 4);
            const uint64_t bd = bd0 + (uint64_t)(((dyi * KC + 2 * kk) * Cfg::KSTEP_BYTES) >> 4);
            umma_bf16(dbase, ad, bd, idesc, (dyi | kk) ? 1u : 0u);
          }
        }
        umma_commit(a_empty + sa);
        umma_commit(c_full + s);
        last = i;
      }
      // the accumulators are freed below: wait (bounded) until the MMAs of the
      // last committed tile, and with them every earlier one, have completed
      if (last >= 0) mbar_wait(a_empty + last % NBUF, (uint32_t)((last / NBUF) & 1), kDrainSpin);
    }
  } else if (warp >= 4) {
    // ---------------- epilogue ---------------------------------------------------------
    // out[x] = b + P_-1[x-1] + P_0[x] + P_+1[x+1]: neighbours within a warp come
    // by shuffles; the lane-0 / lane-31 edges of each 32-pixel quarter go
    // through shared memory (double buffered by tile parity, one named barrier
    // per tile for the epilogue warps).
    const int ew = warp - 4;          // 0 .. NEPI - 1
    const int quarter = warp & 3;     // TMEM lane quarter = pixels 32q .. 32q+31
    const int grp = ew >> 2;          // output-channel group of CG channels
    const int m = quarter * 32 + lane;
    const int x = m & (N - 1);
    const int m0 = quarter * 32;
    const int qleft = ((m0 & (N - 1)) == 0 ? m0 - 1 + N : m0 - 1) >> 5;
    const int qright = (((m0 & (N - 1)) + 32) == N ? m0 + 32 - N : m0 + 32) >> 5;
    int i = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int part = t / npix;
      const int pix = t % npix;
      const int b = pix / tiles_per_img, y0 = (pix % tiles_per_img) * TROWS;
      const int s = i & 1;
      const bool ok = mbar_wait(c_full + s, (i >> 1) & 1, lim);
      if (!ok) atomicOr(a.err, 16u);
      tmem_fence_after_sync();
      const uint32_t tcol = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(s * Cfg::ACC_COLS) + grp * CG;
      float pm[CG], pp[CG], p0[CG];
      float* const eb = bnd + (size_t)s * ((Cfg::NEPI / 4) * 4 * 2 * CG);
      if (ok) {
        tmem_ld_cols<CG>(tcol + 0 * COUT_TILE, pm);
        tmem_ld_cols<CG>(tcol + 2 * COUT_TILE, pp);
        tmem_ld_cols<CG>(tcol + 1 * COUT_TILE, p0);
        tmem_wait_ld();
        float* mine = eb + ((grp * 4 + quarter) * 2) * CG;
        if (Cfg::QR > 1 && lane == 31) {
#pragma unroll
          for (int j = 0; j < CG; ++j) mine[j] = pm[j];
        }
        if (Cfg::QR > 1 && lane == 0) {
#pragma unroll
          for (int j = 0; j < CG; ++j) mine[CG + j] = pp[j];
        }
      }
      // the warps of an exchange group meet once per tile (named barrier 2 + the
      // group's index). The group's abort flag for this tile is written only by
      // its own warps before the barrier and read by them after it, so they all
      // take the same decision; flags alternate with the tile parity, so a warp
      // that already moved on to the next tile never writes the flag its
      // partner is about to read.
      if constexpr (Cfg::QR > 1) {
        const int xg = grp * (4 / Cfg::QR) + quarter / Cfg::QR;
        volatile uint32_t* const flag = pair_abort + (i & 1) * 8 + xg;
        if (!ok) *flag = 1;
        asm volatile("bar.sync %0, %1;" ::"r"(2 + xg), "r"(Cfg::QR * 32) : "memory");
        if (*flag) break;
      } else {
        if (!ok) break;
      }
      const int co0 = a.co_base + part * COUT_TILE + grp * CG;
      const int gy = y0 + m / N;
      const float* eleft = eb + ((grp * 4 + qleft) * 2) * CG;
      const float* eright = eb + ((grp * 4 + qright) * 2) * CG + CG;
      // neighbours by a rotation within the warp; lanes 0 and 31 take the
      // neighbouring quarter's edge value instead (a select, no divergent branch;
      // for N = 32 a quarter is one row and the rotation is already the
      // periodic wrap)
      const bool edge_l = N > 32 && lane == 0, edge_r = N > 32 && lane == 31;
#pragma unroll
      for (int cc = 0; cc < CG; cc += 8) {
        float el[8], er[8];
        if (N > 32) {
#pragma unroll
          for (int j = 0; j < 8; j += 4) {
            const float4 l4 = *reinterpret_cast<const float4*>(eleft + cc + j);
            const float4 r4 = *reinterpret_cast<const float4*>(eright + cc + j);
            el[j] = l4.x, el[j + 1] = l4.y, el[j + 2] = l4.z, el[j + 3] = l4.w;
            er[j] = r4.x, er[j + 1] = r4.y, er[j + 2] = r4.z, er[j + 3] = r4.w;
          }
        }
        float outv[8];
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
          float l0 = __shfl_sync(0xffffffffu, pm[cc + j], (lane + 31) & 31);
          float l1 = __shfl_sync(0xffffffffu, pm[cc + j + 1], (lane + 31) & 31);
          float r0 = __shfl_sync(0xffffffffu, pp[cc + j], (lane + 1) & 31);
          float r1 = __shfl_sync(0xffffffffu, pp[cc + j + 1], (lane + 1) & 31);
          if (N > 32) {
            l0 = edge_l ? el[j] : l0;
            l1 = edge_l ? el[j + 1] : l1;
            r0 = edge_r ? er[j] : r0;
            r1 = edge_r ? er[j + 1] : r1;
          }
          const f32x2 sum = add2(add2(pack2(p0[cc + j], p0[cc + j + 1]), pack2(l0, l1)), pack2(r0, r1));
          unpack2(sum, outv[j], outv[j + 1]);
        }
        const int chunk = (co0 + cc) >> 3;
        const size_t oidx = ((((size_t)b * (a.cout_total / 8) + chunk) * N + gy) * N + x) * 8;
        if (a.gelu == 2) {
          // reverse mode of GELU: multiply by GELU'(pre-activation)
          const uint4 zk = *reinterpret_cast<const uint4*>(a.aux_in + oidx);
          const uint32_t z4[4] = {zk.x, zk.y, zk.z, zk.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&z4[e]));
            outv[2 * e] *= gelu_grad_f(f.x);
            outv[2 * e + 1] *= gelu_grad_f(f.y);
          }
          if (a.dbias) {
            // the layer's bias gradient is the pixel sum of this cotangent: taken
            // here in FP32, before the BF16 rounding of the stored values
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              float sv = outv[j];
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
              if (lane == j) atomicAdd(a.dbias + co0 + cc + j, sv);
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < 8; j += 2) {
            const float2 bb = *reinterpret_cast<const float2*>(sbias + co0 + cc + j);
            unpack2(add2(pack2(outv[j], outv[j + 1]), pack2(bb.x, bb.y)), outv[j], outv[j + 1]);
          }
          if (a.gelu == 1) {
            if (a.aux_out) {
              uint4 zk;
              __nv_bfloat162 z0 = __floats2bfloat162_rn(outv[0], outv[1]);
              __nv_bfloat162 z1 = __floats2bfloat162_rn(outv[2], outv[3]);
              __nv_bfloat162 z2 = __floats2bfloat162_rn(outv[4], outv[5]);
              __nv_bfloat162 z3 = __floats2bfloat162_rn(outv[6], outv[7]);
              zk.x = *reinterpret_cast<uint32_t*>(&z0);
              zk.y = *reinterpret_cast<uint32_t*>(&z1);
              zk.z = *reinterpret_cast<uint32_t*>(&z2);
              zk.w = *reinterpret_cast<uint32_t*>(&z3);
              *reinterpret_cast<uint4*>(a.aux_out + oidx) = zk;
            }
#pragma unroll
            for (int j = 0; j < 8; j += 2) unpack2(gelu2(pack2(outv[j], outv[j + 1])), outv[j], outv[j + 1]);
          }
        }
        uint4 pk;
        __nv_bfloat162 h0 = __floats2bfloat162_rn(outv[0], outv[1]);
        __nv_bfloat162 h1 = __floats2bfloat162_rn(outv[2], outv[3]);
        __nv_bfloat162 h2 = __floats2bfloat162_rn(outv[4], outv[5]);
        __nv_bfloat162 h3 = __floats2bfloat162_rn(outv[6], outv[7]);
        pk.x = *reinterpret_cast<uint32_t*>(&h0);
        pk.y = *reinterpret_cast<uint32_t*>(&h1);
        pk.z = *reinterpret_cast<uint32_t*>(&h2);
        pk.w = *reinterpret_cast<uint32_t*>(&h3);
        *reinterpret_cast<uint4*>(a.out + oidx) = pk;
      }
      tmem_fence_before_sync();
      mbar_arrive(c_empty + s);
    }
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 1) tmem_dealloc(tmem, Cfg::TMEM_COLS);
}

// ---------------------------------------------------------------------------
// First layer (CIN = 2 or 2 k_c, FP32 state input) on CUDA cores:
//   out[p][co] = GELU(b[co] + sum W[co][ci][dy][dx] in[ci][p + (dy, dx)])
// input: state history [k][batch][2][N][N] FP32 (k = CIN / 2 snapshots);
// output: chunk planes [batch][64/8][N][N][8] BF16.
// ---------------------------------------------------------------------------
struct ConvInArgs {
  const float* const* hist;  // device array of CIN/2 pointers to [batch][2][N][N] states
  const float* w;            // [64][CIN][3][3]
  const float* bias;         // [64]
  __nv_bfloat16* out;
  int batch, cin;
};

template <int LOGN>
__global__ void __launch_bounds__(256) conv_in_kernel(const ConvInArgs a) {
  constexpr int N = 1 << LOGN;
  extern __shared__ float sw_in[];  // [64][cin*9] then bias[64]
  const int nw = 64 * a.cin * 9;
  for (int k = threadIdx.x; k < nw; k += blockDim.x) sw_in[k] = a.w[k];
  for (int k = threadIdx.x; k < 64; k += blockDim.x) sw_in[nw + k] = a.bias[k];
  __syncthreads();
  const size_t total = (size_t)a.batch * N * N;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(p / (N * N));
    const int y = (int)((p / N) % N), x = (int)(p % N);
    float in[16][9];
    const int cin = a.cin;
    for (int c = 0; c < cin; ++c) {
      const float* st = a.hist[c >> 1] + ((size_t)b * 2 + (c & 1)) * N * N;
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx)
          in[c][(dy + 1) * 3 + dx + 1] = st[((y + dy) & (N - 1)) * N + ((x + dx) & (N - 1))];
    }
    for (int c8 = 0; c8 < 8; ++c8) {
      float o[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int co = c8 * 8 + j;
        float v = sw_in[nw + co];
        const float* wr = sw_in + co * cin * 9;
        for (int c = 0; c < cin; ++c)
#pragma unroll
          for (int k = 0; k < 9; ++k) v += wr[c * 9 + k] * in[c][k];
        o[j] = gelu_f(v);
      }
      uint4 pk;
      __nv_bfloat162 h0 = __floats2bfloat162_rn(o[0], o[1]);
      __nv_bfloat162 h1 = __floats2bfloat162_rn(o[2], o[3]);
      __nv_bfloat162 h2 = __floats2bfloat162_rn(o[4], o[5]);
      __nv_bfloat162 h3 = __floats2bfloat162_rn(o[6], o[7]);
      pk.x = *reinterpret_cast<uint32_t*>(&h0);
      pk.y = *reinterpret_cast<uint32_t*>(&h1);
      pk.z = *reinterpret_cast<uint32_t*>(&h2);
      pk.w = *reinterpret_cast<uint32_t*>(&h3);
      *reinterpret_cast<uint4*>(a.out + ((((size_t)b * 8 + c8) * N + y) * N + x) * 8) = pk;
    }
  }
}

// ---------------------------------------------------------------------------
// First-layer input for the tensor cores: cin/2 FP32 states -> 16 BF16
// channels per pixel (channels cin .. 15 are zero), chunk planes
// [batch][2][N][N][8].
// ---------------------------------------------------------------------------
struct PackArgs {
  const float* const* hist;  // cin/2 pointers to [batch][2][N][N] states
  const float* single;       // or (cin = 2) the one state directly, when non-null
  __nv_bfloat16* out;        // [batch][2][N][N][8]
  int batch, cin;
};

template <int LOGN>
__global__ void __launch_bounds__(256) pack_input_kernel(const PackArgs a) {
  constexpr int N = 1 << LOGN;
  pdl_wait();
  pdl_trigger();
  const size_t total = (size_t)a.batch * N * N;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(p / (N * N));
    const size_t pix = p % (N * N);
    float v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = 0.f;
    for (int c = 0; c < a.cin; ++c) v[c] = (a.single ? a.single : a.hist[c >> 1])[((size_t)b * 2 + (c & 1)) * N * N + pix];
#pragma unroll
    for (int c8 = 0; c8 < 2; ++c8) {
      uint4 pk;
      __nv_bfloat162 h0 = __floats2bfloat162_rn(v[c8 * 8 + 0], v[c8 * 8 + 1]);
      __nv_bfloat162 h1 = __floats2bfloat162_rn(v[c8 * 8 + 2], v[c8 * 8 + 3]);
      __nv_bfloat162 h2 = __floats2bfloat162_rn(v[c8 * 8 + 4], v[c8 * 8 + 5]);
      __nv_bfloat162 h3 = __floats2bfloat162_rn(v[c8 * 8 + 6], v[c8 * 8 + 7]);
      pk.x = *reinterpret_cast<uint32_t*>(&h0);
      pk.y = *reinterpret_cast<uint32_t*>(&h1);
      pk.z = *reinterpret_cast<uint32_t*>(&h2);
      pk.w = *reinterpret_cast<uint32_t*>(&h3);
      *reinterpret_cast<uint4*>(a.out + (((size_t)b * 2 + c8) * N * N + pix) * 8) = pk;
    }
  }
}

// ---------------------------------------------------------------------------
// Last layer of the temporal-correction network (64 -> 2) on CUDA cores,
// FP32 output [batch][2][N][N] (no activation).
// ---------------------------------------------------------------------------
struct ConvOut2Args {
  const __nv_bfloat16* in;  // [batch][8][N][N][8]
  const float* w;           // [2][64][3][3]
  const float* bias;        // [2]
  float* out;               // [batch][2][N][N]
  int batch;
};

template <int LOGN>
__global__ void __launch_bounds__(256) conv_out2_kernel(const ConvOut2Args a) {
  constexpr int N = 1 << LOGN;
  __shared__ float sw[2 * 64 * 9 + 2];
  for (int k = threadIdx.x; k < 2 * 64 * 9; k += blockDim.x) sw[k] = a.w[k];
  if (threadIdx.x < 2) sw[2 * 64 * 9 + threadIdx.x] = a.bias[threadIdx.x];
  __syncthreads();
  pdl_wait();
  pdl_trigger();
  const size_t total = (size_t)a.batch * N * N;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(p / (N * N));
    const int y = (int)((p / N) % N), x = (int)(p % N);
    float o0 = sw[2 * 64 * 9], o1 = sw[2 * 64 * 9 + 1];
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int yy = (y + dy) & (N - 1), xx = (x + dx) & (N - 1);
        const int k = (dy + 1) * 3 + dx + 1;
        for (int c8 = 0; c8 < 8; ++c8) {
          const uint4 pk = *reinterpret_cast<const uint4*>(a.in + ((((size_t)b * 8 + c8) * N + yy) * N + xx) * 8);
          const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&pk);
#pragma unroll
          for (int j2 = 0; j2 < 4; ++j2) {
            const float2 f = __bfloat1622float2(h[j2]);
            const int c0 = c8 * 8 + 2 * j2;
            o0 += sw[(0 * 64 + c0) * 9 + k] * f.x + sw[(0 * 64 + c0 + 1) * 9 + k] * f.y;
            o1 += sw[(1 * 64 + c0) * 9 + k] * f.x + sw[(1 * 64 + c0 + 1) * 9 + k] * f.y;
          }
        }
      }
    a.out[((size_t)b * 2 + 0) * N * N + y * N + x] = o0;
    a.out[((size_t)b * 2 + 1) * N * N + y * N + x] = o1;
  }
}

}  // namespace ldfv
