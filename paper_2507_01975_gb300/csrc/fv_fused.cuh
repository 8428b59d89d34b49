// fv_fused.cuh -- cluster-resident rollout kernel of the plain FV step.
//
// One thread-block cluster of CS CTAs owns one trajectory of an N x N
// periodic MAC grid for the whole rollout; CTA `rank` owns rows
// [rank*R, (rank+1)*R), R = N / CS, of both velocity components. The state
// never leaves on-chip memory between time steps: the stage state lives in
// shared memory (two buffers, ping-pong, with two halo rows on each side),
// u_n and the RK4 accumulator live in registers of the thread that owns the
// cell, and neighbouring rows and the FFT transposes move through
// distributed shared memory (DSMEM) between the CTAs of the cluster.
//
// Per RK4 stage (App. B.5), for stage state w:
//   1. halo rows of w from the neighbour CTAs (periodic wrap, App. B.1);
//   2. flux block + flux assembly (Sec. 3.4, App. B.2): 4-tap face
//      interpolations/derivatives, advective and diffusive flux differences,
//      Burgers' advective correction, Kolmogorov forcing -> tendency T;
//      acc += b_s T and w' = u_n + a_s dt T (final stage: u_n + dt/6 acc);
//   3. (Navier-Stokes) projection of w' (Sec. 3.6, App. B.3-B.4):
//      cell divergence -> real-to-complex row FFTs (two rows packed per
//      complex transform) -> DSMEM transpose -> column FFTs -> multiply by
//      1 / symbol of D2 G2 (zero mode removed) -> inverse column FFTs ->
//      DSMEM transpose back -> complex-to-real row FFTs -> w' -= G2 p.
#pragma once

#include <cooperative_groups.h>

#include "fv_common.cuh"

namespace ldfv {
namespace cg = cooperative_groups;

struct FvArgs {
  const void* u_in;
  void* u_out;
  void* traj;
  int n_steps;
  int save_every;
  int flow;     // 0 Burgers, 1 Navier-Stokes
  int forcing;  // 0 none, 1 Kolmogorov
  double dt, nu, idx, idy, drag, inv_nn;
  double ci[4], cx[4], cy[4];  // interpolation, x-derivative, y-derivative taps
  const void* tw;    // [N/2] complex: exp(-2 pi i m / N)
  const void* symx;  // [N/2 + 1] Laplacian symbol along x
  const void* symy;  // [N] Laplacian symbol along y
  const void* frc;   // [N] amp sin(kf y_j) at the u-face rows
};

template <typename T, int LOGN, int CS, int NT>
struct FusedCfg {
  static constexpr int N = 1 << LOGN;
  static constexpr int R = N / CS;
  static constexpr int HR = R + 4;
  static constexpr int G = NT / N;
  static constexpr int RT = R / G;
  static constexpr int NC = (CS > 1) ? N / 2 / CS : N / 2;
  static constexpr int COLLEN = N + 1;  // padded column length in the transpose buffer
  static constexpr int KMAX = sizeof(T) == 4 ? 3 : 2;
  using CT = typename Cplx<T>::t;
  static constexpr size_t W_ELEMS = 2 * HR * N;
  static constexpr size_t ROW_CPLX = (size_t)R * (N / 2);
  static constexpr size_t COL_CPLX = (CS > 1) ? (size_t)NC * COLLEN : 0;
  static constexpr size_t OFF_W1 = W_ELEMS * sizeof(T);
  static constexpr size_t OFF_ROW = 2 * W_ELEMS * sizeof(T);
  static constexpr size_t OFF_COL = OFF_ROW + ROW_CPLX * sizeof(CT);
  static constexpr size_t OFF_TW = OFF_COL + COL_CPLX * sizeof(CT);
  static constexpr size_t OFF_SX = OFF_TW + (N / 2) * sizeof(CT);
  static constexpr size_t OFF_SY = OFF_SX + (N / 2 + 2) * sizeof(T);
  static constexpr size_t OFF_FRC = OFF_SY + N * sizeof(T);
  static constexpr size_t SMEM = OFF_FRC + R * sizeof(T);
  static_assert(NT % N == 0, "threads must cover whole rows");
  static_assert(R % G == 0 && RT >= 1, "rows must split evenly over row groups");
  static_assert(R >= 2 && (R % 2) == 0, "each CTA owns an even number of rows >= 2");
  static_assert(CS == 1 || R >= 2, "halo comes from the immediate neighbour");
};

template <int CS>
__device__ __forceinline__ void csync() {
  if constexpr (CS > 1) {
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
}

template <int CS, typename P>
__device__ __forceinline__ P* remote(P* p, int rank) {
  if constexpr (CS > 1) {
    return cg::this_cluster().map_shared_rank(p, (unsigned)rank);
  } else {
    return p;
  }
}

template <typename T, int LOGN, int CS, int NT>
__global__ void __launch_bounds__(NT, 1) fv_rollout_kernel(const FvArgs a) {
  using Cfg = FusedCfg<T, LOGN, CS, NT>;
  using CT = typename Cfg::CT;
  constexpr int N = Cfg::N, R = Cfg::R, HR = Cfg::HR, RT = Cfg::RT, NC = Cfg::NC;
  constexpr int MSK = N - 1;
  extern __shared__ __align__(16) unsigned char smem[];
  T* const wbuf0 = reinterpret_cast<T*>(smem);
  T* const wbuf1 = reinterpret_cast<T*>(smem + Cfg::OFF_W1);
  CT* const rowbuf = reinterpret_cast<CT*>(smem + Cfg::OFF_ROW);
  CT* const colbuf = reinterpret_cast<CT*>(smem + Cfg::OFF_COL);
  CT* const tw = reinterpret_cast<CT*>(smem + Cfg::OFF_TW);
  T* const sx = reinterpret_cast<T*>(smem + Cfg::OFF_SX);
  T* const sy = reinterpret_cast<T*>(smem + Cfg::OFF_SY);
  T* const frc = reinterpret_cast<T*>(smem + Cfg::OFF_FRC);

  const int tid = threadIdx.x;
  int rank = 0;
  if constexpr (CS > 1) rank = (int)cg::this_cluster().block_rank();
  const int prev = (rank + CS - 1) % CS, next = (rank + 1) % CS;
  const int traj = blockIdx.y;
  const int row0 = rank * R;
  const size_t field = (size_t)N * N;

  // ---- constant tables --------------------------------------------------
  for (int k = tid; k < N / 2; k += NT) tw[k] = reinterpret_cast<const CT*>(a.tw)[k];
  for (int k = tid; k <= N / 2; k += NT) sx[k] = reinterpret_cast<const T*>(a.symx)[k];
  for (int k = tid; k < N; k += NT) sy[k] = reinterpret_cast<const T*>(a.symy)[k];
  for (int k = tid; k < R; k += NT) frc[k] = reinterpret_cast<const T*>(a.frc)[row0 + k];

  // ---- initial state: owned rows of u and v ------------------------------
  const T* uin = reinterpret_cast<const T*>(a.u_in) + (size_t)traj * 2 * field;
  for (int e = tid; e < 2 * R * N; e += NT) {
    const int c = e / (R * N), rem = e % (R * N);
    const int r = rem / N, i = rem % N;
    wbuf0[(c * HR + r + 2) * N + i] = uin[c * field + (size_t)(row0 + r) * N + i];
  }
  __syncthreads();

  const int ci = tid % N;
  const int jr0 = (tid / N) * RT;
  T un[2][RT], acc[2][RT];
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int r = 0; r < RT; ++r) un[c][r] = wbuf0[(c * HR + jr0 + r + 2) * N + ci];

  const T dt = (T)a.dt, nu = (T)a.nu, idx = (T)a.idx, idy = (T)a.idy, drag = (T)a.drag;
  const T inv_nn = (T)a.inv_nn;
  T kci[4], kcx[4], kcy[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    kci[q] = (T)a.ci[q];
    kcx[q] = (T)a.cx[q];
    kcy[q] = (T)a.cy[q];
  }
  const bool ns = a.flow == 1;
  const bool forced = a.forcing == 1;

  int cur = 0;
  int snap = 0;
  for (int step = 1; step <= a.n_steps; ++step) {
#pragma unroll 1
    for (int stage = 0; stage < 4; ++stage) {
      T* const wr = cur ? wbuf1 : wbuf0;
      T* const ww = cur ? wbuf0 : wbuf1;

      // 1. halo rows of the stage state from the neighbour CTAs
      csync<CS>();
      {
        const T* wp = remote<CS>(wr, prev);
        const T* wn = remote<CS>(wr, next);
        for (int e = tid; e < 8 * N; e += NT) {
          const int c = e / (4 * N), rem = e % (4 * N);
          const int h = rem / N, i = rem % N;
          if (h < 2) {
            wr[(c * HR + h) * N + i] = wp[(c * HR + R + h) * N + i];
          } else {
            wr[(c * HR + R + h) * N + i] = wn[(c * HR + h) * N + i];
          }
        }
      }
      __syncthreads();

      // 2. tendency, RK4 combination
      {
        const T* fu = wr;
        const T* fv = wr + HR * N;
        auto ax = [&](const T* f, int hr, int i0, const T* k) -> T {
          const T* row = f + hr * N;
          return k[0] * row[i0 & MSK] + k[1] * row[(i0 + 1) & MSK] + k[2] * row[(i0 + 2) & MSK] +
                 k[3] * row[(i0 + 3) & MSK];
        };
        auto ay = [&](const T* f, int hr0, int i, const T* k) -> T {
          const int ii = i & MSK;
          return k[0] * f[hr0 * N + ii] + k[1] * f[(hr0 + 1) * N + ii] + k[2] * f[(hr0 + 2) * N + ii] +
                 k[3] * f[(hr0 + 3) * N + ii];
        };
        const T ca = stage == 2 ? dt : (T)0.5 * dt;
#pragma unroll
        for (int r = 0; r < RT; ++r) {
          const int hr = jr0 + r + 2;
          const int i = ci;
          const T Uc0 = ax(fu, hr, i - 1, kci), Uc1 = ax(fu, hr, i - 2, kci);
          const T Gxc0 = ax(fu, hr, i - 1, kcx), Gxc1 = ax(fu, hr, i - 2, kcx);
          const T Uk0 = ay(fu, hr - 2, i, kci), Uk1 = ay(fu, hr - 1, i, kci);
          const T Gyu0 = ay(fu, hr - 2, i, kcy), Gyu1 = ay(fu, hr - 1, i, kcy);
          const T Vk0 = ax(fv, hr, i - 2, kci), Vk1 = ax(fv, hr + 1, i - 2, kci);
          const T UkR = ay(fu, hr - 2, i + 1, kci), VkR = ax(fv, hr, i - 1, kci);
          const T Gxv0 = ax(fv, hr, i - 2, kcx), GxvR = ax(fv, hr, i - 1, kcx);
          const T Vc0 = ay(fv, hr - 1, i, kci), VcS = ay(fv, hr - 2, i, kci);
          const T Gyc0 = ay(fv, hr - 1, i, kcy), GycS = ay(fv, hr - 2, i, kcy);
          T tu = -(Uc0 * Uc0 - Uc1 * Uc1) * idx - (Uk1 * Vk1 - Uk0 * Vk0) * idy +
                 nu * ((Gxc0 - Gxc1) * idx + (Gyu1 - Gyu0) * idy);
          T tv = -(UkR * VkR - Uk0 * Vk0) * idx - (Vc0 * Vc0 - VcS * VcS) * idy +
                 nu * ((GxvR - Gxv0) * idx + (Gyc0 - GycS) * idy);
          const T uc = fu[hr * N + i], vc = fv[hr * N + i];
          if (!ns) {
            const T divc0 = Gxc0 + Gyc0;
            const T divcW = Gxc1 + ay(fv, hr - 1, i - 1, kcy);
            const T divcS = ax(fu, hr - 1, i - 1, kcx) + GycS;
            tu += uc * (T)0.5 * (divcW + divc0);
            tv += vc * (T)0.5 * (divcS + divc0);
          }
          if (forced) {
            tu += frc[jr0 + r] - drag * uc;
            tv += -drag * vc;
          }
          T nu_, nv_;
          if (stage == 0) {
            acc[0][r] = tu;
            acc[1][r] = tv;
          } else if (stage < 3) {
            acc[0][r] += (T)2 * tu;
            acc[1][r] += (T)2 * tv;
          }
          if (stage < 3) {
            nu_ = un[0][r] + ca * tu;
            nv_ = un[1][r] + ca * tv;
          } else {
            const T c6 = dt / (T)6;
            nu_ = un[0][r] + c6 * (acc[0][r] + tu);
            nv_ = un[1][r] + c6 * (acc[1][r] + tv);
          }
          ww[hr * N + i] = nu_;
          ww[(HR + hr) * N + i] = nv_;
        }
      }

      // 3. projection of the new stage state
      if (ns) {
        csync<CS>();
        {  // v row just above the owned rows, for the divergence of the last row
          const T* wn = remote<CS>(ww, next);
          for (int i = tid; i < N; i += NT) ww[(HR + R + 2) * N + i] = wn[(HR + 2) * N + i];
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < RT; ++r) {
          const int jj = jr0 + r, hr = jj + 2;
          const T* fu = ww + hr * N;
          const T* fv = ww + HR * N;
          const T d = (fu[(ci + 1) & MSK] - fu[ci]) * idx + (fv[(hr + 1) * N + ci] - fv[hr * N + ci]) * idy;
          T* z = reinterpret_cast<T*>(&rowbuf[(jj >> 1) * N + ci]);
          z[jj & 1] = d;
        }
        __syncthreads();
        // forward row transforms: R/2 complex rows of length N
        fft_dif<CT, LOGN, Cfg::KMAX, 0, false>(rowbuf, R / 2, N, 1, tw, tid, NT);
        // unpack two real rows per complex row into half spectra [R][N/2]
        // (entry 0 packs the real DC and Nyquist values as re + i im)
        {
          constexpr int TOT = (R / 2) * (N / 2);
          constexpr int IT = (TOT + NT - 1) / NT;
          CT A[IT], B[IT];
#pragma unroll
          for (int it = 0; it < IT; ++it) {
            const int item = tid + it * NT;
            if (item < TOT) {
              const int jp = item / (N / 2), k = item % (N / 2);
              const CT* Z = rowbuf + jp * N;
              if (k == 0) {
                const CT z0 = Z[0], zh = Z[1];  // bit-reversed positions of 0 and N/2
                A[it] = CT{z0.x, zh.x};
                B[it] = CT{z0.y, zh.y};
              } else {
                const CT zk = Z[brev<LOGN>(k)], zm = Z[brev<LOGN>(N - k)];
                A[it] = CT{(T)0.5 * (zk.x + zm.x), (T)0.5 * (zk.y - zm.y)};
                B[it] = CT{(T)0.5 * (zk.y + zm.y), (T)-0.5 * (zk.x - zm.x)};
              }
            }
          }
          __syncthreads();
#pragma unroll
          for (int it = 0; it < IT; ++it) {
            const int item = tid + it * NT;
            if (item < TOT) {
              const int jp = item / (N / 2), k = item % (N / 2);
              rowbuf[(2 * jp) * (N / 2) + k] = A[it];
              rowbuf[(2 * jp + 1) * (N / 2) + k] = B[it];
            }
          }
          __syncthreads();
        }
        // column transforms, spectral multiply, inverse column transforms
        CT* cb;
        int cSS, cES;
        if constexpr (CS > 1) {
          csync<CS>();
          for (int e = tid; e < NC * N; e += NT) {
            const int kxl = e % NC, ky = e / NC;
            const CT* src = remote<CS>(rowbuf, ky / R);
            colbuf[kxl * Cfg::COLLEN + ky] = src[(ky % R) * (N / 2) + rank * NC + kxl];
          }
          __syncthreads();
          cb = colbuf;
          cSS = Cfg::COLLEN;
          cES = 1;
          fft_dif<CT, LOGN, Cfg::KMAX, 0, false>(cb, NC, cSS, cES, tw, tid, NT);
        } else {
          cb = rowbuf;
          cSS = 1;
          cES = N / 2;
          fft_dif<CT, LOGN, Cfg::KMAX, 0, true>(cb, NC, cSS, cES, tw, tid, NT);
        }
        for (int e = tid; e < NC * N; e += NT) {
          const int kxl = e % NC, pos = e / NC;
          const int kx = rank * NC + kxl;
          const int ky = brev<LOGN>(pos);
          if (kx != 0) {
            CT& z = cb[kxl * cSS + pos * cES];
            const T m = inv_nn / (sx[kx] + sy[ky]);
            z = CT{z.x * m, z.y * m};
          } else if (ky <= N / 2) {
            // packed column: DC column in the real part, Nyquist column in
            // the imaginary part; both real and even in ky.
            const int kyb = (N - ky) & MSK;
            CT& zk = cb[pos * cES];
            CT& zm = cb[brev<LOGN>(kyb) * cES];
            const T m0 = ky == 0 ? (T)0 : inv_nn / (sx[0] + sy[ky]);
            const T mn = inv_nn / (sx[N / 2] + sy[ky]);
            const T hp = (T)0.5 * (m0 + mn), hm = (T)0.5 * (m0 - mn);
            const CT a0 = zk, b0 = zm;
            zk = CT{hp * a0.x + hm * b0.x, hp * a0.y - hm * b0.y};
            if (kyb != ky) zm = CT{hp * b0.x + hm * a0.x, hp * b0.y - hm * a0.y};
          }
        }
        __syncthreads();
        if constexpr (CS > 1) {
          fft_dit<CT, LOGN, Cfg::KMAX, 0, false>(cb, NC, cSS, cES, tw, tid, NT);
          csync<CS>();
          for (int e = tid; e < R * (N / 2); e += NT) {
            const int r = e % R, kx = e / R;
            const CT* src = remote<CS>(colbuf, kx / NC);
            rowbuf[r * (N / 2) + kx] = src[(kx % NC) * Cfg::COLLEN + row0 + r];
          }
          __syncthreads();
        } else {
          fft_dit<CT, LOGN, Cfg::KMAX, 0, true>(cb, NC, cSS, cES, tw, tid, NT);
        }
        // repack half spectra into complex rows (bit-reversed) and invert
        {
          constexpr int TOT = (R / 2) * (N / 2);
          constexpr int IT = (TOT + NT - 1) / NT;
          CT Z0[IT], Z1[IT];
#pragma unroll
          for (int it = 0; it < IT; ++it) {
            const int item = tid + it * NT;
            if (item < TOT) {
              const int jp = item / (N / 2), k = item % (N / 2);
              const CT A = rowbuf[(2 * jp) * (N / 2) + k];
              const CT B = rowbuf[(2 * jp + 1) * (N / 2) + k];
              if (k == 0) {
                Z0[it] = CT{A.x, B.x};
                Z1[it] = CT{A.y, B.y};
              } else {
                Z0[it] = CT{A.x - B.y, A.y + B.x};
                Z1[it] = CT{A.x + B.y, B.x - A.y};
              }
            }
          }
          __syncthreads();
#pragma unroll
          for (int it = 0; it < IT; ++it) {
            const int item = tid + it * NT;
            if (item < TOT) {
              const int jp = item / (N / 2), k = item % (N / 2);
              CT* Z = rowbuf + jp * N;
              if (k == 0) {
                Z[0] = Z0[it];
                Z[1] = Z1[it];
              } else {
                Z[brev<LOGN>(k)] = Z0[it];
                Z[brev<LOGN>(N - k)] = Z1[it];
              }
            }
          }
          __syncthreads();
        }
        fft_dit<CT, LOGN, Cfg::KMAX, 0, false>(rowbuf, R / 2, N, 1, tw, tid, NT);
        // pressure rows are ready in every CTA: w' -= G2 p
        csync<CS>();
        {
          const T* pl = reinterpret_cast<const T*>(rowbuf);
          const T* pp = reinterpret_cast<const T*>(remote<CS>(rowbuf, prev));
          auto pat = [&](const T* base, int jj, int i) -> T {
            return base[((jj >> 1) * N + (i & MSK)) * 2 + (jj & 1)];
          };
#pragma unroll
          for (int r = 0; r < RT; ++r) {
            const int jj = jr0 + r, hr = jj + 2;
            const T pc = pat(pl, jj, ci);
            const T pw = pat(pl, jj, ci - 1);
            const T ps = jj > 0 ? pat(pl, jj - 1, ci) : pat(pp, R - 1, ci);
            ww[hr * N + ci] -= (pc - pw) * idx;
            ww[(HR + hr) * N + ci] -= (pc - ps) * idy;
          }
        }
      }
      cur ^= 1;
    }

    // end of the time step: the current buffer holds u_{n+1}
    const T* wc = cur ? wbuf1 : wbuf0;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int r = 0; r < RT; ++r) un[c][r] = wc[(c * HR + jr0 + r + 2) * N + ci];
    if (a.save_every > 0 && a.traj != nullptr && (step % a.save_every) == 0) {
      T* out = reinterpret_cast<T*>(a.traj) + ((size_t)snap * gridDim.y + traj) * 2 * field;
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int r = 0; r < RT; ++r) out[c * field + (size_t)(row0 + jr0 + r) * N + ci] = un[c][r];
      ++snap;
    }
  }

  T* uout = reinterpret_cast<T*>(a.u_out) + (size_t)traj * 2 * field;
  const T* wc = cur ? wbuf1 : wbuf0;
  (void)wc;
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int r = 0; r < RT; ++r) uout[c * field + (size_t)(row0 + jr0 + r) * N + ci] = un[c][r];
  // keep every CTA of the cluster resident until all DSMEM reads are done
  csync<CS>();
}

}  // namespace ldfv
