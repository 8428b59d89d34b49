// conv_wgrad.cuh -- weight and bias gradients of a periodic 3x3 convolution
// on the tensor cores (tcgen05, BF16 operands, FP32 accumulation in TMEM).
//
// For a layer out[o][p] = b[o] + sum_{c,dy,dx} W[o][c][dy][dx] h[c][p + (dy,dx)]
// with output cotangent z[o][p], the reverse mode gives
//   dW[o][c][dy][dx] = sum_{b,p} z[o][p] h[c][p + (dy,dx)],   db[o] = sum_{b,p} z[o][p],
// a contraction over every pixel of the batch (K = batch x N x N).
//
// Both activations are stored as chunk planes [batch][C/8][N][N][8] BF16.
// Eight consecutive pixels of one plane are 128 contiguous bytes = one
// MN-major core matrix (8 K-rows x 8 channels), so the planes are the MMA
// operands as they are: A = h (M = channels), B = z (N = output channels),
// K = 16 pixels of one image row per instruction. In shared memory every h
// row carries a periodic x-halo ([row][c8][N + 2][16 B]), so the dx shift is a
// 16-byte start-address offset; the dy shift picks the row. With CIN = 64,
// M = 128 covers two consecutive h rows (taps dy and dy + 1) and two MMAs per
// dx cover dy = -1, 0 (| +1, +2 unused); with CIN = 16, one M = 128 MMA covers
// rows dy = -1 .. 6 (only -1 .. 1 used). Each CTA accumulates its share of
// the pixels in TMEM and writes FP32 partial sums; a second kernel reduces
// them over the CTAs and adds them to the gradient array (deterministic).
//
// Roles: warp 0 (all lanes) issues the bulk copies of the next item's rows,
// warp 1 allocates TMEM and its lane 0 issues the MMAs, warps 4..7 sum the
// z tiles for the bias gradient and read the accumulators out at the end.
// Every mbarrier wait is bounded and records an error on time-out.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "conv_tc.cuh"

namespace ldfv {

struct WgradArgs {
  const __nv_bfloat16* h;  // layer input [batch][CIN/8][N][N][8]
  const __nv_bfloat16* z;  // output cotangent [batch][cout_total/8][N][N][8]
  float* partial;          // [parts][gx][3 dx][NMMA][O_TILE][128 lanes]
  float* partial_b;        // [parts][gx][O_TILE]
  int batch;
  int cout_total;
  unsigned* err;
  long long spin_limit;
};

template <int LOGN, int CIN, int O_TILE>
struct WgradCfg {
  static constexpr int N = 1 << LOGN;
  static constexpr int P = N + 2;                 // pixels per staged h row (periodic halo)
  static constexpr int KC = CIN / 8;
  static constexpr int OC8 = O_TILE / 8;
  static constexpr int RPM = 128 / CIN;           // h rows covered by one M = 128 operand
  static constexpr int NMMA = (3 + RPM - 1) / RPM;
  static constexpr int R = 256 / N;               // output rows per work item
  static constexpr int HR = R + NMMA * RPM - 1;   // staged h rows per item
  static constexpr uint32_t HROW_BYTES = KC * P * 16;
  static constexpr uint32_t H_BYTES = HR * HROW_BYTES;
  static constexpr uint32_t ZROW_BYTES = OC8 * N * 16;
  static constexpr uint32_t Z_BYTES = R * ZROW_BYTES;
  static constexpr uint32_t STAGE_BYTES = align16(H_BYTES + Z_BYTES);
  static constexpr uint32_t OFF_BAR = 2 * STAGE_BYTES;
  static constexpr uint32_t SMEM = OFF_BAR + 128;
  static constexpr int ACC_COLS = 3 * NMMA * O_TILE;
  static constexpr int TMEM_COLS = ACC_COLS <= 256 ? 256 : 512;
  static constexpr int NT = 256;
  static constexpr int NBIAS = 128;               // warps 4..7
  static_assert(CIN == 16 || CIN == 64, "input channels");
  static_assert(O_TILE % 16 == 0 && O_TILE <= 256, "MMA N");
  static_assert(ACC_COLS <= 512, "tensor memory");
  static_assert(SMEM <= 232448, "shared memory");
  static_assert(N >= 32 && N <= 128, "row length");
  static_assert(OC8 * 16 <= 2 * NBIAS, "bias threads");
};

template <int LOGN, int CIN, int O_TILE>
__global__ void __launch_bounds__(256, 1) conv_wgrad_kernel(const WgradArgs a) {
  using Cfg = WgradCfg<LOGN, CIN, O_TILE>;
  constexpr int N = Cfg::N, P = Cfg::P, KC = Cfg::KC, OC8 = Cfg::OC8, R = Cfg::R, HR = Cfg::HR;
  constexpr int RPM = Cfg::RPM, NMMA = Cfg::NMMA;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* const bars = reinterpret_cast<uint64_t*>(smem + Cfg::OFF_BAR);
  uint64_t* const full = bars + 0;   // [2]
  uint64_t* const empty = bars + 2;  // [2]
  uint64_t* const done = bars + 4;
  uint32_t* const tslot = reinterpret_cast<uint32_t*>(bars + 5);
  volatile uint32_t* const abort_flag = reinterpret_cast<volatile uint32_t*>(bars + 6);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int part = blockIdx.y;
  const int gx = gridDim.x;
  const int items_per_img = N / R;
  const int nitems = a.batch * items_per_img;
  const long long lim = a.spin_limit;
  const int zc0 = part * OC8;  // first 8-channel chunk of this part in z

  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1 + Cfg::NBIAS);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tslot, Cfg::TMEM_COLS);
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tmem = *tslot;
  pdl_wait();
  pdl_trigger();

  if (warp == 0) {
    // ---------------- producer: h rows with periodic halo, z rows -------------------
    int i = 0, issued = 0;
    for (int it = blockIdx.x; it < nitems; it += gx, ++i) {
      const int b = it / items_per_img, y0 = (it % items_per_img) * R;
      const int s = i & 1;
      int ok = 1;
      if (lane == 0) ok = mbar_wait(empty + s, ((i >> 1) & 1) ^ 1, lim) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) {
          *abort_flag = 1;
          atomicOr(a.err, 32u);
        }
        break;
      }
      if (lane == 0) mbar_expect_tx(full + s, (uint32_t)(HR * KC * P * 16 + R * OC8 * N * 16));
      __syncwarp();
      unsigned char* const hs = smem + s * Cfg::STAGE_BYTES;
      unsigned char* const zs = hs + Cfg::H_BYTES;
      // h: HR rows x KC chunks, three copies each (row body, left and right halo)
      for (int k = lane; k < HR * KC * 3; k += 32) {
        const int piece = k % 3, rc = k / 3;
        const int r = rc / KC, c = rc % KC;
        const int gy = (y0 - 1 + r) & (N - 1);
        const unsigned char* src = reinterpret_cast<const unsigned char*>(a.h) + ((((size_t)b * KC + c) * N + gy) * N) * 16;
        unsigned char* dst = hs + (r * KC + c) * P * 16;
        if (piece == 0)
          bulk_g2s(dst + 16, src, N * 16, full + s);
        else if (piece == 1)
          bulk_g2s(dst, src + (N - 1) * 16, 16, full + s);
        else
          bulk_g2s(dst + (N + 1) * 16, src, 16, full + s);
      }
      for (int k = lane; k < R * OC8; k += 32) {
        const int t = k / OC8, c = k % OC8;
        const unsigned char* src = reinterpret_cast<const unsigned char*>(a.z) +
                                   ((((size_t)b * (a.cout_total / 8) + zc0 + c) * N + y0 + t) * N) * 16;
        bulk_g2s(zs + (t * OC8 + c) * N * 16, src, N * 16, full + s);
      }
      issued = i + 1;
    }
    // never leave with copies in flight
    if (lane == 0)
      for (int j = issued - 2; j < issued; ++j)
        if (j >= 0) mbar_wait(full + (j & 1), (j >> 1) & 1, kDrainSpin);
  } else if (warp == 1) {
    // ---------------- MMA issuer ------------------------------------------------------
    if (lane == 0) {
      constexpr uint32_t idesc = umma_idesc_bf16<128, O_TILE>() | (1u << 15) | (1u << 16);  // A, B MN-major
      int i = 0;
      bool first = true;
      for (int it = blockIdx.x; it < nitems; it += gx, ++i) {
        const int s = i & 1;
        if (*abort_flag) break;
        if (!mbar_wait(full + s, (i >> 1) & 1, lim)) {
          *abort_flag = 1;
          atomicOr(a.err, 64u);
          break;
        }
        tmem_fence_after_sync();
        const uint32_t hb = smem_u32(smem + s * Cfg::STAGE_BYTES);
        const uint32_t zb = hb + Cfg::H_BYTES;
        // base descriptors; each MMA adds a constant to the start address field
        const uint64_t ad0 = umma_desc(hb, 128, P * 16);
        const uint64_t bd0 = umma_desc(zb, 128, N * 16);
#pragma unroll 1
        for (int t = 0; t < R; ++t) {
#pragma unroll
          for (int dx = 0; dx < 3; ++dx) {
#pragma unroll
            for (int mm = 0; mm < NMMA; ++mm) {
              const uint32_t d = tmem + (uint32_t)((dx * NMMA + mm) * O_TILE);
#pragma unroll
              for (int kc = 0; kc < N / 16; ++kc) {
                // h rows (y - 1 + mm RPM) .., pixels 16 kc + dx - 1 (+1 for the halo)
                const uint64_t ad =
                    ad0 + (uint64_t)((((t + mm * RPM) * Cfg::HROW_BYTES) + (16 * kc + dx) * 16) >> 4);
                const uint64_t bd = bd0 + (uint64_t)((t * Cfg::ZROW_BYTES + 16 * kc * 16) >> 4);
                umma_bf16(d, ad, bd, idesc, (first && t == 0 && kc == 0) ? 0u : 1u);
              }
            }
          }
        }
        first = false;
        umma_commit(empty + s);
      }
      umma_commit(done);
      // tensor memory is freed below: wait (bounded) for every MMA issued here
      mbar_wait(done, 0, kDrainSpin);
    }
  } else if (warp >= 4) {
    // ---------------- bias sums during the loop, accumulator read-out at the end ------
    const int bt = tid - 128;  // 0..127
    float accb[2][8];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int j = 0; j < 8; ++j) accb[u][j] = 0.f;
    int i = 0;
    bool fail = false;
    for (int it = blockIdx.x; it < nitems; it += gx, ++i) {
      const int s = i & 1;
      if (!mbar_wait(full + s, (i >> 1) & 1, lim)) {
        fail = true;
        atomicOr(a.err, 128u);
        break;
      }
      const unsigned char* zs = smem + s * Cfg::STAGE_BYTES + Cfg::H_BYTES;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int w = bt + 128 * u;  // (chunk, pixel residue mod 16)
        if (w < OC8 * 16) {
          const int c = w >> 4, sub = w & 15;
          for (int t = 0; t < R; ++t)
            for (int x = sub; x < N; x += 16) {
              const uint4 v = *reinterpret_cast<const uint4*>(zs + ((t * OC8 + c) * N + x) * 16);
              const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w4[e]));
                accb[u][2 * e] += f.x;
                accb[u][2 * e + 1] += f.y;
              }
            }
        }
      }
      mbar_arrive(empty + s);
    }
    // reduce over the 16 pixel residues (16 consecutive threads share a chunk)
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) accb[u][j] += __shfl_xor_sync(0xffffffffu, accb[u][j], o);
    float* pb = a.partial_b + ((size_t)part * gx + blockIdx.x) * O_TILE;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int w = bt + 128 * u;
      if (w < OC8 * 16 && (w & 15) == 0)
#pragma unroll
        for (int j = 0; j < 8; ++j) pb[(w >> 4) * 8 + j] = accb[u][j];
    }
    // accumulators: lane quarter (warp & 3), columns (dx, mm, o)
    const bool ok = !fail && mbar_wait(done, 0, lim);
    if (!ok) atomicOr(a.err, 256u);
    tmem_fence_after_sync();
    const int quarter = warp & 3;
    const int m = quarter * 32 + lane;
    float* pp = a.partial + ((size_t)part * gx + blockIdx.x) * (size_t)(3 * NMMA * O_TILE * 128);
    const bool any = (int)blockIdx.x < nitems;
#pragma unroll 1
    for (int col = 0; col < Cfg::ACC_COLS; col += 8) {
      float v[8];
      if (ok && any) {
        tmem_ld8_nowait(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)col, v);
        tmem_wait_ld();
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = 0.f;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) pp[(size_t)(col + j) * 128 + m] = v[j];
    }
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 1) tmem_dealloc(tmem, Cfg::TMEM_COLS);
}

// Sum the per-CTA partials and add them to the gradient of a layer stored as
// W[cout][cin][3][3] and b[cout] (FP32), output channels co_base + part * O_TILE + o.
struct WgradReduceArgs {
  const float* partial;
  const float* partial_b;
  float* dW;
  float* db;
  int gx, parts, cin, co_base;
  int cout_real;  // output channels of the layer: tile channels at or beyond it carry padding
};

template <int CIN, int O_TILE>
__global__ void __launch_bounds__(256) conv_wgrad_reduce_kernel(const WgradReduceArgs a) {
  constexpr int RPM = 128 / CIN, NMMA = (3 + RPM - 1) / RPM;
  const int nw = a.parts * O_TILE * a.cin * 9;
  const size_t cta_stride = (size_t)3 * NMMA * O_TILE * 128;
  pdl_wait();
  pdl_trigger();
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nw + a.parts * O_TILE; e += gridDim.x * blockDim.x) {
    if (e < nw) {
      // e enumerates (part, o, a, dx, c) with c fastest: coalesced partial reads
      const int c = e % a.cin;
      const int dx = (e / a.cin) % 3;
      const int ay = (e / (a.cin * 3)) % 3;  // dy + 1
      const int o = (e / (a.cin * 9)) % O_TILE;
      const int part = e / (a.cin * 9 * O_TILE);
      const int mm = ay / RPM, lane = (ay % RPM) * CIN + c;
      const float* src = a.partial + (size_t)part * a.gx * cta_stride + (size_t)((dx * NMMA + mm) * O_TILE + o) * 128 + lane;
      float s = 0.f;
      for (int x = 0; x < a.gx; ++x) s += src[(size_t)x * cta_stride];
      const int co = a.co_base + part * O_TILE + o;
      if (co < a.cout_real) a.dW[(((size_t)co * a.cin + c) * 3 + ay) * 3 + dx] += s;
    } else {
      const int k = e - nw;
      const int part = k / O_TILE, o = k % O_TILE;
      float s = 0.f;
      for (int x = 0; x < a.gx; ++x) s += a.partial_b[((size_t)part * a.gx + x) * O_TILE + o];
      if (a.db && a.co_base + part * O_TILE + o < a.cout_real) a.db[a.co_base + part * O_TILE + o] += s;
    }
  }
}

}  // namespace ldfv
