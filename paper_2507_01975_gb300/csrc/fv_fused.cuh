// fv_fused.cuh -- cluster-resident rollout kernel of the plain FV step.
//
// One thread-block cluster of CS CTAs owns one trajectory of an N x N
// periodic MAC grid for the whole rollout; CTA `rank` owns rows
// [rank*R, (rank+1)*R), R = N / CS, of both velocity components. The stage
// state lives in shared memory with two halo rows below and three above; the
// state at the start of the time step (u_n) and the RK4 accumulator live in
// tensor memory (TMEM), in the lane of the thread that owns the cell.
// Neighbouring rows and the FFT transposes move through distributed shared
// memory (DSMEM). Global memory is touched only to load the initial state and
// to store snapshots and the final state.
//
// Per RK4 stage (App. B.5), for stage state w:
//   A. cluster barrier, halo rows of w from the neighbour CTAs (periodic
//      wrap, App. B.1);
//   C. flux block + flux assembly (Sec. 3.4, App. B.2): 4-tap face
//      interpolations/derivatives, advective and diffusive flux differences,
//      Burgers' advective correction, Kolmogorov forcing -> tendency T;
//      acc += b_s T and w' = u_n + a_s dt T (final stage: u_n + dt/6 acc).
//      The CTA also recomputes v' on the first row of the next CTA, so the
//      divergence of its last row needs no extra exchange;
//   D. (Navier-Stokes) projection of w' (Sec. 3.6, App. B.3-B.4): cell
//      divergence computed in registers -> warp FFTs of two real rows packed
//      as one complex row, unpacked into half spectra -> DSMEM transpose ->
//      warp column FFTs, multiply by 1 / symbol of D2 G2 (zero mode removed),
//      inverse column FFTs -> DSMEM transpose back -> inverse warp row FFTs ->
//      w' -= G2 p (the row below comes from the previous CTA through DSMEM).
//      The transposes are in place through registers (two cluster barriers
//      each), except at N = 256, where the transforms store their outputs
//      straight into the owning CTAs' buffers (one barrier each).
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
  int traj_batch;  // trajectories per snapshot in traj (0: the launch's batch)
  int flow;     // 0 Burgers, 1 Navier-Stokes
  int forcing;  // 0 none, 1 Kolmogorov
  double dt, nu, idx, idy, drag, inv_nn;
  const void* tw;    // [N/2] complex: exp(-2 pi i m / N)
  const void* symx;  // [N/2 + 1] Laplacian symbol along x
  const void* symy;  // [N] Laplacian symbol along y
  const void* frc;   // [N] amp sin(kf y_j) at the u-face rows
};

template <typename T, int LOGN, int CS, int NT>
struct FusedCfg {
  static constexpr int N = 1 << LOGN;
  static constexpr int R = N / CS;
  static constexpr int HR = R + 5;  // 2 halo rows below, 3 above
  static constexpr int G = NT / N;
  static constexpr int RT = R / G;
  static constexpr int NW = NT / 32;
  static constexpr int NC = N / 2 / CS;  // spectral columns owned after the transpose
  // N = 256: the FFTs are warp-level Stockham transforms with an exchange
  // buffer per warp (WarpFFT256), and the transposes are fused into them: the
  // forward row transforms store their half spectra straight into the owning
  // CTAs' column buffers, the inverse column transforms theirs straight into
  // the owning CTAs' row buffers (remote stores, one cluster barrier each).
  // Smaller N keep the shuffle transforms and the in-place transposes.
  static constexpr bool STOCK = LOGN == 8 && sizeof(T) == 4;
  static constexpr int COLLEN = N + 1;   // padded column length
  static constexpr int HSTR = N / 2 + 1; // padded half-spectrum row length
  using CT = typename Cplx<T>::t;
  using FFT = WarpFFT<T, LOGN>;
  static constexpr size_t W_BYTES = (size_t)2 * HR * N * sizeof(T);
  static constexpr size_t ROW_BYTES = (size_t)R * HSTR * sizeof(CT);
  static constexpr size_t COL_BYTES = (size_t)NC * COLLEN * sizeof(CT);
  static constexpr size_t PR_BYTES = (size_t)R * 2 * HSTR * sizeof(T);
  // fused transposes (N = 256): the buffers a warp's remote stores fill are
  // laid out so that the 32 lanes of one store write contiguous bytes --
  // half spectra by spectral column, hsT[kx][RSTR] (the two rows of one
  // inverse row transform are adjacent: one 16-byte load), and columns by
  // row, colT[ky][NCP]; the pressure rows reuse the column buffer
  static constexpr int RSTR = R + 2;
  static constexpr int NCP = NC + 1;
  static constexpr size_t HST_BYTES = (size_t)(N / 2) * RSTR * sizeof(CT);
  static constexpr size_t COLT_BYTES = cmax((size_t)N * NCP * sizeof(CT), PR_BYTES);
  // rows and columns share one buffer for the in-place transposes
  static constexpr size_t SCR_BYTES =
      STOCK ? align16(HST_BYTES) + align16(COLT_BYTES) : align16(cmax(ROW_BYTES, COL_BYTES));
  static constexpr size_t OFF_SCR = align16(W_BYTES);
  static constexpr size_t OFF_COL = STOCK ? OFF_SCR + align16(HST_BYTES) : OFF_SCR;
  static constexpr size_t OFF_TW = OFF_SCR + SCR_BYTES;
  static constexpr size_t OFF_SX = OFF_TW + align16((N / 2) * sizeof(CT));
  static constexpr size_t OFF_SY = OFF_SX + align16((N / 2 + 2) * sizeof(T));
  static constexpr size_t OFF_FRC = OFF_SY + align16(N * sizeof(T));
  static constexpr size_t OFF_ROW0 = OFF_FRC + align16(R * sizeof(T));  // u_n.v and acc.v of row 0
  static constexpr size_t OFF_TMEM = OFF_ROW0 + align16(2 * N * sizeof(T));
  // N = 256: the tendency phase works on strips of 4 cells (register window,
  // strip_tendency); GC row groups of N/4 strips, RTC bands per CTA
  static constexpr int GC = NT / (N / 4), RTC = R / GC;
  static constexpr size_t OFF_XB = OFF_TMEM + 16;
  static constexpr size_t XB_BYTES = STOCK ? (size_t)NW * WarpFFT256<T>::XB * sizeof(CT) : 0;
  static constexpr size_t SMEM = OFF_XB + XB_BYTES;
  // forward-transpose and backward-transpose register staging per thread
  static constexpr int NFWD = (NC * N + NT - 1) / NT;
  static constexpr int NBWD = (R * (N / 2) + NT - 1) / NT;
  // one CTA per SM: the full 128-register budget (no spills) is worth more than
  // fitting a second CTA, which measured slower on the 256^2 batch
  static constexpr int MIN_BLOCKS = 1;
  // TMEM: RT rows x (u_n.u, u_n.v, acc.u, acc.v) per thread; warps sharing a
  // lane quarter take consecutive column ranges
  static constexpr int SLOT = CellSlot<T>::COLS;
  static constexpr int TCOLS_THREAD = RT * SLOT;
  static constexpr int TCOLS_NEED = ((NW + 3) / 4) * TCOLS_THREAD;
  static constexpr int TMEM_COLS = TCOLS_NEED <= 32 ? 32 : TCOLS_NEED <= 64 ? 64 : TCOLS_NEED <= 128 ? 128
                                 : TCOLS_NEED <= 256 ? 256 : 512;
  static_assert(TCOLS_NEED <= 512, "per-thread state exceeds tensor memory");
  // clustered configurations must never wait for TMEM: at most two CTAs per SM
  // fit by shared memory or registers, and two of them still fit in 512 columns
  static_assert(CS == 1 || 2 * TMEM_COLS <= 512, "co-resident clusters must never wait for TMEM");
  static_assert(NT % N == 0, "threads must cover whole rows");
  static_assert(R % G == 0 && RT >= 1, "rows must split evenly over row groups");
  static_assert(G >= 2, "in-place band update needs at least two row groups");
  static_assert(R >= 4 && (R % 2) == 0, "each CTA owns an even number of rows >= 4");
  static_assert(NT % 32 == 0, "whole warps");
};

// fast division for the FP32 spectral multiply (2 ulp), exact for FP64
__device__ __forceinline__ float sdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double sdiv(double a, double b) { return a / b; }

template <int CS>
__device__ __forceinline__ void csync() {
  if constexpr (CS > 1) {
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
}

// split cluster barrier: every thread arrives once and then waits once
template <int CS>
__device__ __forceinline__ void cluster_arrive() {
  if constexpr (CS > 1) asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
template <int CS>
__device__ __forceinline__ void cluster_wait() {
  if constexpr (CS > 1) asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <int CS, typename P>
__device__ __forceinline__ P* remote(P* p, int rank) {
  if constexpr (CS > 1) {
    return cg::this_cluster().map_shared_rank(p, (unsigned)rank);
  } else {
    return p;
  }
}

// Tendency H(w) at u-face (hr, i) and v-face (hr, i) of the padded tile
// (App. B.2 advection, dissipation and forcing terms) with the fixed physics
// kernels of App. B.2: linear interpolation [0, 1/2, 1/2, 0] and the
// derivative [1, -27, 27, -1] / 24h (DORD = 4) or [0, -1, 1, 0] / h (DORD = 2).
template <typename T, int N, int DORD>
struct Tendency {
  const T* fu;
  const T* fv;
  T idx, idy, nu, drag;
  bool burgers, forced;

  // taps f0..f3 at axial offsets -3/2, -1/2, 1/2, 3/2
  static __device__ __forceinline__ T ip(T f1, T f2) { return (T)0.5 * (f1 + f2); }
  static __device__ __forceinline__ T dv(T f0, T f1, T f2, T f3, T ih) {
    if constexpr (DORD == 4) {
      return ((f0 - f3) + (T)27 * (f2 - f1)) * (ih * (T)(1.0 / 24.0));
    } else {
      return (f2 - f1) * ih;
    }
  }
  __device__ __forceinline__ T at(const T* f, int hr, int i) const { return f[hr * N + (i & (N - 1))]; }
  // along x, output half a cell after tap i0 + 1
  __device__ __forceinline__ T ix(const T* f, int hr, int i0) const { return ip(at(f, hr, i0 + 1), at(f, hr, i0 + 2)); }
  __device__ __forceinline__ T dx(const T* f, int hr, int i0) const {
    return dv(at(f, hr, i0), at(f, hr, i0 + 1), at(f, hr, i0 + 2), at(f, hr, i0 + 3), idx);
  }
  __device__ __forceinline__ T iy(const T* f, int hr0, int i) const { return ip(at(f, hr0 + 1, i), at(f, hr0 + 2, i)); }
  __device__ __forceinline__ T dy(const T* f, int hr0, int i) const {
    return dv(at(f, hr0, i), at(f, hr0 + 1, i), at(f, hr0 + 2, i), at(f, hr0 + 3, i), idy);
  }
  __device__ __forceinline__ void eval(int hr, int i, T fx, T& tu, T& tv) const {
    const T Uc0 = ix(fu, hr, i - 1), Uc1 = ix(fu, hr, i - 2);
    const T Gxc0 = dx(fu, hr, i - 1), Gxc1 = dx(fu, hr, i - 2);
    const T Uk0 = iy(fu, hr - 2, i), Uk1 = iy(fu, hr - 1, i);
    const T Gyu0 = dy(fu, hr - 2, i), Gyu1 = dy(fu, hr - 1, i);
    const T Vk0 = ix(fv, hr, i - 2), Vk1 = ix(fv, hr + 1, i - 2);
    const T UkR = iy(fu, hr - 2, i + 1), VkR = ix(fv, hr, i - 1);
    const T Gxv0 = dx(fv, hr, i - 2), GxvR = dx(fv, hr, i - 1);
    const T Vc0 = iy(fv, hr - 1, i), VcS = iy(fv, hr - 2, i);
    const T Gyc0 = dy(fv, hr - 1, i), GycS = dy(fv, hr - 2, i);
    tu = -(Uc0 * Uc0 - Uc1 * Uc1) * idx - (Uk1 * Vk1 - Uk0 * Vk0) * idy +
         nu * ((Gxc0 - Gxc1) * idx + (Gyu1 - Gyu0) * idy);
    tv = -(UkR * VkR - Uk0 * Vk0) * idx - (Vc0 * Vc0 - VcS * VcS) * idy +
         nu * ((GxvR - Gxv0) * idx + (Gyc0 - GycS) * idy);
    const T uc = at(fu, hr, i), vc = at(fv, hr, i);
    if (burgers) {
      const T divc0 = Gxc0 + Gyc0;
      const T divcW = Gxc1 + dy(fv, hr - 1, i - 1);
      const T divcS = dx(fu, hr - 1, i - 1) + GycS;
      tu += uc * (T)0.5 * (divcW + divc0);
      tv += vc * (T)0.5 * (divcS + divc0);
    }
    if (forced) {
      tu += fx - drag * uc;
      tv += -drag * vc;
    }
  }
};

// The rollout of trajectory `traj` of a.u_in by the calling CTA (its cluster's
// share of the rows), with this CTA's tensor memory at tmem_base (TMEM_COLS
// columns allocated by the caller). Every thread of the CTA calls it; it starts
// by overwriting the whole shared-memory layout and ends with a cluster-wide
// barrier, so consecutive calls need no synchronisation between them.
template <typename T, int LOGN, int CS, int NT, int DORD>
__device__ __forceinline__ void fv_rollout_body(const FvArgs& a, int traj, uint32_t tmem_base) {
  using Cfg = FusedCfg<T, LOGN, CS, NT>;
  using CT = typename Cfg::CT;
  using FFT = typename Cfg::FFT;
  using Slot = CellSlot<T>;
  constexpr int N = Cfg::N, R = Cfg::R, HR = Cfg::HR, RT = Cfg::RT, NC = Cfg::NC, NW = Cfg::NW;
  constexpr int HALF = N / 2, HSTR = Cfg::HSTR;
  constexpr int MSK = N - 1;
  constexpr int W = FFT::W, E = FFT::E, TPW = 32 / W;
  extern __shared__ __align__(1024) unsigned char smem[];
  T* const wt = reinterpret_cast<T*>(smem);  // [2][HR][N]
  unsigned char* const scr = smem + Cfg::OFF_SCR;
  // half spectra (rows): [R][HSTR], N = 256: hsT [N/2][RSTR]
  CT* const hs = reinterpret_cast<CT*>(scr);
  // columns: [NC][COLLEN], N = 256: colT [N][NCP]
  CT* const col = reinterpret_cast<CT*>(smem + Cfg::OFF_COL);
  // pressure rows [R][2 HSTR] (over the half spectra, N = 256: over the columns)
  T* const pr = reinterpret_cast<T*>(Cfg::STOCK ? smem + Cfg::OFF_COL : scr);
  CT* const tw = reinterpret_cast<CT*>(smem + Cfg::OFF_TW);
  T* const sx = reinterpret_cast<T*>(smem + Cfg::OFF_SX);
  T* const sy = reinterpret_cast<T*>(smem + Cfg::OFF_SY);
  T* const frc = reinterpret_cast<T*>(smem + Cfg::OFF_FRC);
  T* const unrow0 = reinterpret_cast<T*>(smem + Cfg::OFF_ROW0);  // u_n.v on local row 0
  T* const accrow0 = unrow0 + N;                                // acc.v on local row 0 (stage 2)
  CT* const xbuf = reinterpret_cast<CT*>(smem + Cfg::OFF_XB);  // [NW][288] (N = 256 only)

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int q = lane & (W - 1), gbase = lane & ~(W - 1);
  int rank = 0;
  if constexpr (CS > 1) rank = (int)cg::this_cluster().block_rank();
  const int prev = (rank + CS - 1) % CS, next = (rank + 1) % CS;
  const int row0 = rank * R;
  const size_t NN = (size_t)N * N;

  for (int k = tid; k < HALF; k += NT) tw[k] = reinterpret_cast<const CT*>(a.tw)[k];
  for (int k = tid; k <= HALF; k += NT) sx[k] = reinterpret_cast<const T*>(a.symx)[k];
  for (int k = tid; k < N; k += NT) sy[k] = reinterpret_cast<const T*>(a.symy)[k];
  for (int k = tid; k < R; k += NT) frc[k] = reinterpret_cast<const T*>(a.frc)[row0 + k];

  const T* uin = reinterpret_cast<const T*>(a.u_in) + (size_t)traj * 2 * NN;
  T* uout = reinterpret_cast<T*>(a.u_out) + (size_t)traj * 2 * NN;
  for (int e = tid; e < 2 * R * N; e += NT) {
    const int c = e / (R * N), rem = e % (R * N);
    const int r = rem / N, i = rem % N;
    wt[(c * HR + r + 2) * N + i] = uin[c * NN + (size_t)(row0 + r) * N + i];
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  // this thread's TMEM slots: lane quarter of the warp, column range of the warp
  const uint32_t tbase = tmem_base + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * Cfg::TCOLS_THREAD);

  const int ci = tid % N;
  const int grp = tid / N;
  const bool ns = a.flow == 1;
  Tendency<T, N, DORD> tend;
  tend.fu = wt;
  tend.fv = wt + HR * N;
  tend.idx = (T)a.idx;
  tend.idy = (T)a.idy;
  tend.nu = (T)a.nu;
  tend.drag = (T)a.drag;
  tend.burgers = a.flow == 0;
  tend.forced = a.forcing == 1;
  const T dt = (T)a.dt, idx = (T)a.idx, idy = (T)a.idy, inv_nn = (T)a.inv_nn;
  const bool extra = ns && (grp == Cfg::G - 1);  // recompute v' on the next CTA's first row

  // u_n of the owned cells into TMEM (N = 256: the cells of the thread's strips)
  const int sx4 = 4 * (tid % (N / 4)), gc = tid / (N / 4);
  auto store_un = [&]() {
    if constexpr (Cfg::STOCK) {
      // the strips' cells were last written by other threads (gradient phase)
      __syncthreads();
#pragma unroll
      for (int r = 0; r < Cfg::RTC; ++r) {
        const int hr = r * Cfg::GC + gc + 2;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          Slot::store(tbase + (4 * r + q) * Cfg::SLOT, wt[hr * N + sx4 + q], wt[(HR + hr) * N + sx4 + q], (T)0, (T)0);
      }
    } else {
#pragma unroll
      for (int r = 0; r < RT; ++r) {
        const int hr = r * Cfg::G + grp + 2;
        Slot::store(tbase + r * Cfg::SLOT, wt[hr * N + ci], wt[(HR + hr) * N + ci], (T)0, (T)0);
      }
    }
  };
  store_un();
  if (grp == 0) unrow0[ci] = wt[(HR + 2) * N + ci];
  tmem_wait_st();

  // Halo exchange by pushes (N = 256, Navier-Stokes): at the end of every
  // stage each CTA stores its first three rows into the previous CTA's halo
  // rows above and its last two rows into the next CTA's halo rows below, then
  // arrives on the cluster barrier; the next stage starts with the matching
  // wait. No CTA reads another's state rows, so phase C updates its rows in
  // place without waiting for the neighbours. The pushes land after the
  // neighbours' last reads of those halo rows (phases C and D1 of the same
  // stage, behind two cluster barriers since).
  const bool fused = Cfg::STOCK && ns;
  auto push_halos = [&]() {
    T* wp = remote<CS>(wt, prev);
    T* wn = remote<CS>(wt, next);
    constexpr int Q = N / 4;  // float4 per row
    for (int e = tid; e < 10 * Q; e += NT) {
      const int c = e / (5 * Q), rem = e % (5 * Q);
      const int h = rem / Q, i = 4 * (rem % Q);
      if (h < 3) {  // rows 2 + h -> the previous CTA's rows R + 2 + h
        *reinterpret_cast<float4*>(wp + (c * HR + R + 2 + h) * N + i) =
            *reinterpret_cast<const float4*>(wt + (c * HR + 2 + h) * N + i);
      } else {  // rows R + h - 3 -> the next CTA's rows h - 3
        *reinterpret_cast<float4*>(wn + (c * HR + h - 3) * N + i) =
            *reinterpret_cast<const float4*>(wt + (c * HR + R + h - 3) * N + i);
      }
    }
  };
  if (fused) {
    push_halos();
    cluster_arrive<CS>();
  }

  int snap = 0;
  for (int step = 1; step <= a.n_steps; ++step) {
#pragma unroll 1
    for (int stage = 0; stage < 4; ++stage) {
      // ---- A: halo rows -----------------------------------------------------
      if (fused) {
        cluster_wait<CS>();  // the neighbours' pushes of the previous stage landed
      } else {
        csync<CS>();
        const T* wp = remote<CS>(wt, prev);
        const T* wn = remote<CS>(wt, next);
        for (int e = tid; e < 10 * N; e += NT) {
          const int c = e / (5 * N), rem = e % (5 * N);
          const int h = rem / N, i = rem % N;
          if (h < 2) {
            wt[(c * HR + h) * N + i] = wp[(c * HR + R + h) * N + i];
          } else {
            wt[(c * HR + R + h) * N + i] = wn[(c * HR + h) * N + i];
          }
        }
        // the neighbours read this CTA's rows above; phase C overwrites them in
        // place, so its first write waits until every CTA of the cluster has
        // arrived here (split barrier: the wait falls after two bands of work)
        cluster_arrive<CS>();
      }
      __syncthreads();

      // ---- C: tendency and RK4 combination -------------------------------------
      // Rows are processed in bands of G rows (band r = rows r G .. r G + G - 1,
      // one per row group) by all threads in lockstep. Band r reads rows
      // r G - 2 .. r G + G + 1, so once every thread has finished band r, band
      // r - 1 is never read again and its new values are written in place.
      if constexpr (Cfg::STOCK) {
        // strips: thread (gc, strip) owns rows r GC + gc at columns sx4 .. sx4 + 3;
        // bands of GC rows in lockstep, band r - 1 written after band r (as below)
        constexpr int GC = Cfg::GC, RTC = Cfg::RTC;
        const T ca = stage == 2 ? dt : (T)0.5 * dt;
        const T c6 = dt / (T)6;
        const bool xtra = ns && (gc == GC - 1);  // v' on the next CTA's first row
        auto window = [&](int hr, T (&u)[5][8], T (&v)[5][8]) {
#pragma unroll
          for (int rr = 0; rr < 5; ++rr) {
            const T* ru = wt + (hr - 2 + rr) * N;
            const T* rv = wt + (HR + hr - 2 + rr) * N;
            const float2 lu = *reinterpret_cast<const float2*>(ru + ((sx4 - 2) & MSK));
            const float4 mu = *reinterpret_cast<const float4*>(ru + sx4);
            const float2 gu = *reinterpret_cast<const float2*>(ru + ((sx4 + 4) & MSK));
            const float2 lv = *reinterpret_cast<const float2*>(rv + ((sx4 - 2) & MSK));
            const float4 mv = *reinterpret_cast<const float4*>(rv + sx4);
            const float2 gv = *reinterpret_cast<const float2*>(rv + ((sx4 + 4) & MSK));
            u[rr][0] = lu.x; u[rr][1] = lu.y; u[rr][2] = mu.x; u[rr][3] = mu.y;
            u[rr][4] = mu.z; u[rr][5] = mu.w; u[rr][6] = gu.x; u[rr][7] = gu.y;
            v[rr][0] = lv.x; v[rr][1] = lv.y; v[rr][2] = mv.x; v[rr][3] = mv.y;
            v[rr][4] = mv.z; v[rr][5] = mv.w; v[rr][6] = gv.x; v[rr][7] = gv.y;
          }
        };
        T pu[4], pv[4], wve[4];
#pragma unroll
        for (int r = 0; r < RTC; ++r) {
          const int jj = r * GC + gc, hr = jj + 2;
          uint32_t tr[4][4];
#pragma unroll
          for (int q = 0; q < 4; ++q) tmem_ld4(tbase + (4 * r + q) * Cfg::SLOT, tr[q]);
          T u[5][8], v[5][8];
          window(hr, u, v);
          T tu[4], tv[4];
          strip_tendency<T, DORD>(u, v, idx, idy, tend.nu, tend.burgers, tend.forced, frc[jj], tend.drag, tu, tv);
          tmem_wait_ld();
          T nu4[4], nv4[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const T unu = __uint_as_float(tr[q][0]), unv = __uint_as_float(tr[q][1]);
            T au = __uint_as_float(tr[q][2]), av = __uint_as_float(tr[q][3]);
            if (stage == 0) {
              au = tu[q];
              av = tv[q];
            } else if (stage < 3) {
              au += (T)2 * tu[q];
              av += (T)2 * tv[q];
            } else {
              au += tu[q];
              av += tv[q];
            }
            if (stage < 3) {
              Slot::store(tbase + (4 * r + q) * Cfg::SLOT, unu, unv, au, av);
              nu4[q] = unu + ca * tu[q];
              nv4[q] = unv + ca * tv[q];
              if (stage == 2 && jj == 0) accrow0[sx4 + q] = av;
            } else {
              nu4[q] = unu + c6 * au;
              nv4[q] = unv + c6 * av;
            }
          }
          if (r == RTC - 1 && xtra) {
            // v' on the next CTA's first row, from rows R-2 .. R+2
            const T* nrow = remote<CS>(unrow0, next);
            T ue[5][8], ve[5][8];
            window(R + 2, ue, ve);
            T eu[4], ev[4];
            strip_tendency<T, DORD>(ue, ve, idx, idy, tend.nu, tend.burgers, tend.forced, (T)0, tend.drag, eu, ev);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const T unv0 = nrow[sx4 + q];
              wve[q] = stage < 3 ? unv0 + ca * ev[q] : unv0 + c6 * (nrow[N + sx4 + q] + ev[q]);
            }
          }
          __syncthreads();
          if (r == 1 && !fused) cluster_wait<CS>();
          if (r > 0) {
            const int hp = (r - 1) * GC + gc + 2;
            *reinterpret_cast<float4*>(wt + hp * N + sx4) = make_float4(pu[0], pu[1], pu[2], pu[3]);
            *reinterpret_cast<float4*>(wt + (HR + hp) * N + sx4) = make_float4(pv[0], pv[1], pv[2], pv[3]);
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            pu[q] = nu4[q];
            pv[q] = nv4[q];
          }
        }
        tmem_wait_st();
        if constexpr (RTC == 1) {
          if (!fused) cluster_wait<CS>();
        }
        __syncthreads();
        const int hl = (RTC - 1) * GC + gc + 2;
        *reinterpret_cast<float4*>(wt + hl * N + sx4) = make_float4(pu[0], pu[1], pu[2], pu[3]);
        *reinterpret_cast<float4*>(wt + (HR + hl) * N + sx4) = make_float4(pv[0], pv[1], pv[2], pv[3]);
        if (xtra)
          *reinterpret_cast<float4*>(wt + (HR + R + 2) * N + sx4) = make_float4(wve[0], wve[1], wve[2], wve[3]);
        __syncthreads();
      } else
      {
        const T ca = stage == 2 ? dt : (T)0.5 * dt;
        const T c6 = dt / (T)6;
        T pu = (T)0, pv = (T)0, wv_extra = (T)0;
#pragma unroll
        for (int r = 0; r < RT; ++r) {
          const int jj = r * Cfg::G + grp, hr = jj + 2;
          const uint32_t ta = tbase + r * Cfg::SLOT;
          T unu, unv, au, av;
          Slot::load(ta, unu, unv, au, av);
          T tu, tv;
          tend.eval(hr, ci, frc[jj], tu, tv);
          if (stage == 0) {
            au = tu;
            av = tv;
          } else if (stage < 3) {
            au += (T)2 * tu;
            av += (T)2 * tv;
          } else {
            au += tu;
            av += tv;
          }
          T nu_, nv_;
          if (stage < 3) {
            Slot::store(ta, unu, unv, au, av);
            nu_ = unu + ca * tu;
            nv_ = unv + ca * tv;
            if (stage == 2 && jj == 0) accrow0[ci] = av;
          } else {
            nu_ = unu + c6 * au;
            nv_ = unv + c6 * av;
          }
          if (r == RT - 1 && extra) {
            // v' on the next CTA's first row, from rows R-2 .. R+2
            const T* nrow = remote<CS>(unrow0, next);
            T eu, ev;
            tend.eval(R + 2, ci, (T)0, eu, ev);
            const T unv0 = nrow[ci];
            wv_extra = stage < 3 ? unv0 + ca * ev : unv0 + c6 * (nrow[N + ci] + ev);
          }
          __syncthreads();
          if (r == 1) cluster_wait<CS>();
          if (r > 0) {
            const int hp = (r - 1) * Cfg::G + grp + 2;
            wt[hp * N + ci] = pu;
            wt[(HR + hp) * N + ci] = pv;
          }
          pu = nu_;
          pv = nv_;
        }
        tmem_wait_st();
        if constexpr (RT == 1) cluster_wait<CS>();
        __syncthreads();
        const int hl = (RT - 1) * Cfg::G + grp + 2;
        wt[hl * N + ci] = pu;
        wt[(HR + hl) * N + ci] = pv;
        if (extra) wt[(HR + R + 2) * N + ci] = wv_extra;
        __syncthreads();
      }

      if (ns) {
        // ---- D1: divergence, forward row FFTs, half spectra ---------------------
        // half-spectrum rows hold kx in natural order for N = 256 (Stockham)
        // and bit-reversed order otherwise; column 0 packs kx = 0 and N/2
        if constexpr (Cfg::STOCK) {
          using F2 = WarpFFT256<T>;
          const T* fu = wt;
          const T* fv = wt + HR * N;
          CT* xb = xbuf + warp * F2::XB;
          for (int pp = warp; pp < R / 2; pp += NW) {
            const int ja = 2 * pp, hra = ja + 2, hrb = ja + 3;
            CT z[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) {
              const int x = lane + 32 * m;
              const T da = (fu[hra * N + ((x + 1) & MSK)] - fu[hra * N + x]) * idx +
                           (fv[(hra + 1) * N + x] - fv[hra * N + x]) * idy;
              const T db = (fu[hrb * N + ((x + 1) & MSK)] - fu[hrb * N + x]) * idx +
                           (fv[(hrb + 1) * N + x] - fv[hrb * N + x]) * idy;
              z[m] = CT{da, db};
            }
            F2::forward(z, xb, tw, lane);
#pragma unroll
            for (int i = 0; i < 8; ++i) xb[F2::pad(F2::out_index(lane, i))] = z[i];
            __syncwarp();
            // two real rows from one complex transform: A_k = (Z_k + conj Z_{N-k}) / 2,
            // B_k = (Z_k - conj Z_{N-k}) / (2i); k = 0 packs the DC and Nyquist values
            for (int k = lane; k < HALF; k += 32) {
              const CT zk = xb[F2::pad(k)];
              const CT zm = xb[F2::pad(k == 0 ? HALF : N - k)];
              CT A, B;
              if (k == 0) {
                A = CT{zk.x, zm.x};
                B = CT{zk.y, zm.y};
              } else {
                A = CT{(T)0.5 * (zk.x + zm.x), (T)0.5 * (zk.y - zm.y)};
                B = CT{(T)0.5 * (zk.y + zm.y), (T)-0.5 * (zk.x - zm.x)};
              }
              // rows ja, ja + 1 of spectral column k, owned by CTA k / NC
              CT* dst = remote<CS>(col, k / NC) + (row0 + ja) * Cfg::NCP + (k % NC);
              dst[0] = A;
              dst[Cfg::NCP] = B;
            }
            __syncwarp();
          }
        } else {
          const T* fu = wt;
          const T* fv = wt + HR * N;
          for (int t0 = warp * TPW; t0 < R / 2; t0 += NW * TPW) {
            const int jp = t0 + lane / W;
            const bool act = jp < R / 2;
            const int ja = act ? 2 * jp : 0;
            CT z[E];
#pragma unroll
            for (int m = 0; m < E; ++m) {
              const int x = q + W * m;
              const int hra = ja + 2, hrb = ja + 3;
              const T da = (fu[hra * N + ((x + 1) & MSK)] - fu[hra * N + x]) * idx +
                           (fv[(hra + 1) * N + x] - fv[hra * N + x]) * idy;
              const T db = (fu[hrb * N + ((x + 1) & MSK)] - fu[hrb * N + x]) * idx +
                           (fv[(hrb + 1) * N + x] - fv[hrb * N + x]) * idy;
              z[m] = CT{da, db};
            }
            FFT::dif(z, q, tw);
#pragma unroll
            for (int m = 0; m < E; ++m) {
              const int k = brev<LOGN>(q + W * m);
              const int pl = (k == 0) ? 1 : FFT::partner_lane(q, m);
              const CT zm = shfl_idx(z[FFT::partner_reg(m)], gbase + pl);
              const CT zk = z[m];
              CT A, B;
              if (k == 0) {
                A = CT{zk.x, zm.x};
                B = CT{zk.y, zm.y};
              } else {
                A = CT{(T)0.5 * (zk.x + zm.x), (T)0.5 * (zk.y - zm.y)};
                B = CT{(T)0.5 * (zk.y + zm.y), (T)-0.5 * (zk.x - zm.x)};
              }
              const CT Bo = shfl_up1(B);
              const int s = (q + W * m) >> 1;
              if (act) {
                if ((q & 1) == 0)
                  hs[ja * HSTR + s] = A;
                else
                  hs[(ja + 1) * HSTR + s] = Bo;
              }
            }
          }
        }
        csync<CS>();
        // ---- D2: transpose rows -> columns (in place, through registers) --------
        if constexpr (!Cfg::STOCK) {
          CT reg[Cfg::NFWD];
#pragma unroll
          for (int k = 0; k < Cfg::NFWD; ++k) {
            const int e = tid + k * NT;
            if (e < NC * N) {
              const int sl = e % NC, ky = e / NC;
              const CT* src = remote<CS>(hs, ky / R);
              reg[k] = src[(ky % R) * HSTR + rank * NC + sl];
            }
          }
          csync<CS>();
#pragma unroll
          for (int k = 0; k < Cfg::NFWD; ++k) {
            const int e = tid + k * NT;
            if (e < NC * N) {
              const int sl = e % NC, ky = e / NC;
              col[sl * Cfg::COLLEN + ky] = reg[k];
            }
          }
          __syncthreads();
        }
        // ---- D3: column FFTs, spectral multiply, inverse column FFTs -----------
        if constexpr (Cfg::STOCK) {
          using F2 = WarpFFT256<T>;
          CT* xb = xbuf + warp * F2::XB;
          for (int sl = warp; sl < NC; sl += NW) {
            const int kx = rank * NC + sl;  // natural order; column 0 packs kx = 0 and N/2
            CT z[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) z[m] = col[(lane + 32 * m) * Cfg::NCP + sl];
            F2::forward(z, xb, tw, lane);
#pragma unroll
            for (int i = 0; i < 8; ++i) xb[F2::pad(F2::out_index(lane, i))] = z[i];
            __syncwarp();
            // multiply by 1 / (N^2 L(kx, ky)) while gathering the inverse's input
            // pattern; column 0: Z'[ky] = hp Z[ky] + hm conj(Z[-ky]) (kx = 0 in the
            // real part, kx = N/2 in the imaginary part, both real and even in ky)
#pragma unroll
            for (int m = 0; m < 8; ++m) {
              const int ky = lane + 32 * m;
              const CT za = xb[F2::pad(ky)];
              if (kx != 0) {
                const T ma = sdiv(inv_nn, sx[kx] + sy[ky]);
                z[m] = CT{za.x * ma, za.y * ma};
              } else {
                const CT pa = xb[F2::pad((N - ky) & MSK)];
                const T m0 = ky == 0 ? (T)0 : sdiv(inv_nn, sx[0] + sy[ky]);
                const T mn = sdiv(inv_nn, sx[HALF] + sy[ky]);
                const T hp = (T)0.5 * (m0 + mn), hm = (T)0.5 * (m0 - mn);
                z[m] = CT{hp * za.x + hm * pa.x, hp * za.y - hm * pa.y};
              }
            }
            __syncwarp();
            F2::inverse(z, xb, tw, lane);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              // row ky of spectral column kx, owned by CTA ky / R
              const int ky = F2::out_index(lane, i);
              remote<CS>(hs, ky / R)[kx * Cfg::RSTR + (ky % R)] = z[i];
            }
          }
        } else {
        for (int t0 = warp * TPW; t0 < NC; t0 += NW * TPW) {
          const int sl = t0 + lane / W;
          const bool act = sl < NC;
          const int slc = act ? sl : 0;
          const int sg = rank * NC + slc;
          const int kx = brev<LOGN - 1>(sg);
          CT z[E];
#pragma unroll
          for (int m = 0; m < E; ++m) z[m] = col[slc * Cfg::COLLEN + q + W * m];
          FFT::dif(z, q, tw);
          // multiply by 1 / (N^2 L(kx, ky)). Column sg = 0 packs kx = 0 in the
          // real part and kx = N/2 in the imaginary part (both real and even
          // in ky): Z'[ky] = hp Z[ky] + hm conj(Z[-ky]). Registers m and
          // partner_reg(m) hold partner elements, so pairs update in place.
          // All lanes of the warp take part in the shuffles.
#pragma unroll
          for (int m = 0; m < E; ++m) {
            const int mp = FFT::partner_reg(m);
            if (mp < m) continue;
            const int ky = brev<LOGN>(q + W * m);
            const int kyp = brev<LOGN>(q + W * mp);
            const CT za = z[m], zb = z[mp];
            const CT pa = shfl_idx(zb, gbase + FFT::partner_lane(q, m));   // Z[-ky]
            const CT pb = shfl_idx(za, gbase + FFT::partner_lane(q, mp));  // Z[-kyp]
            if (sg != 0) {
              const T ma = sdiv(inv_nn, sx[kx] + sy[ky]);
              const T mb = sdiv(inv_nn, sx[kx] + sy[kyp]);
              z[m] = CT{za.x * ma, za.y * ma};
              if (mp != m) z[mp] = CT{zb.x * mb, zb.y * mb};
            } else {
              {
                const T m0 = ky == 0 ? (T)0 : sdiv(inv_nn, sx[0] + sy[ky]);
                const T mn = sdiv(inv_nn, sx[HALF] + sy[ky]);
                const T hp = (T)0.5 * (m0 + mn), hm = (T)0.5 * (m0 - mn);
                z[m] = CT{hp * za.x + hm * pa.x, hp * za.y - hm * pa.y};
              }
              if (mp != m) {
                const T m0 = kyp == 0 ? (T)0 : sdiv(inv_nn, sx[0] + sy[kyp]);
                const T mn = sdiv(inv_nn, sx[HALF] + sy[kyp]);
                const T hp = (T)0.5 * (m0 + mn), hm = (T)0.5 * (m0 - mn);
                z[mp] = CT{hp * zb.x + hm * pb.x, hp * zb.y - hm * pb.y};
              }
            }
          }
          FFT::dit_inv(z, q, tw);
          if (act) {
#pragma unroll
            for (int m = 0; m < E; ++m) col[slc * Cfg::COLLEN + q + W * m] = z[m];
          }
        }
        }
        csync<CS>();
        // ---- D4: transpose columns -> rows (in place) ---------------------------
        if constexpr (!Cfg::STOCK) {
          CT reg[Cfg::NBWD];
#pragma unroll
          for (int k = 0; k < Cfg::NBWD; ++k) {
            const int e = tid + k * NT;
            if (e < R * HALF) {
              const int rr = e % R, s = e / R;
              const CT* src = remote<CS>(col, s / NC);
              reg[k] = src[(s % NC) * Cfg::COLLEN + row0 + rr];
            }
          }
          csync<CS>();
#pragma unroll
          for (int k = 0; k < Cfg::NBWD; ++k) {
            const int e = tid + k * NT;
            if (e < R * HALF) {
              const int rr = e % R, s = e / R;
              hs[rr * HSTR + s] = reg[k];
            }
          }
          __syncthreads();
        }
        // ---- D5: inverse row FFTs -> pressure rows -------------------------------
        if constexpr (Cfg::STOCK) {
          using F2 = WarpFFT256<T>;
          CT* xb = xbuf + warp * F2::XB;
          for (int pp = warp; pp < R / 2; pp += NW) {
            const int ra = 2 * pp;
            // packed transform Z_k = A_k + i B_k of rows ra, ra + 1 from the
            // half spectra (natural order, column 0 packing DC and Nyquist)
            CT z[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) {
              const int k = lane + 32 * m;
              const int kp = N - k;  // in (0, N/2] for k >= N/2
              const int ks = k < HALF ? k : (kp == HALF ? 0 : kp);
              const float4 ab = *reinterpret_cast<const float4*>(hs + ks * Cfg::RSTR + ra);
              const CT A = CT{ab.x, ab.y}, B = CT{ab.z, ab.w};
              if (k < HALF)
                z[m] = (k == 0) ? CT{A.x, B.x} : CT{A.x - B.y, A.y + B.x};
              else
                z[m] = (kp == HALF) ? CT{A.y, B.y} : CT{A.x + B.y, B.x - A.y};
            }
            F2::inverse(z, xb, tw, lane);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int x = F2::out_index(lane, i);
              pr[ra * (2 * HSTR) + x] = z[i].x;
              pr[(ra + 1) * (2 * HSTR) + x] = z[i].y;
            }
          }
        } else {
        for (int t0 = warp * TPW; t0 < R / 2; t0 += NW * TPW) {
          const int jp = t0 + lane / W;
          const bool act = jp < R / 2;
          const int ra = act ? 2 * jp : 0;
          CT z[E];
#pragma unroll
          for (int m = 0; m < E; ++m) {
            const int p = q + W * m;
            const int k = brev<LOGN>(p);
            if (k < HALF) {
              const CT A = hs[ra * HSTR + (p >> 1)];
              const CT B = hs[(ra + 1) * HSTR + (p >> 1)];
              z[m] = (k == 0) ? CT{A.x, B.x} : CT{A.x - B.y, A.y + B.x};
            } else {
              const int kp = N - k;  // in (0, N/2]
              const int sp = brev<LOGN>(kp & MSK) >> 1;
              const CT A = hs[ra * HSTR + sp];
              const CT B = hs[(ra + 1) * HSTR + sp];
              z[m] = (kp == HALF) ? CT{A.y, B.y} : CT{A.x + B.y, B.x - A.y};
            }
          }
          FFT::dit_inv(z, q, tw);
          __syncwarp();
          if (act) {
#pragma unroll
            for (int m = 0; m < E; ++m) {
              const int x = q + W * m;
              pr[ra * (2 * HSTR) + x] = z[m].x;
              pr[(ra + 1) * (2 * HSTR) + x] = z[m].y;
            }
          }
        }
        }
        // pressure of the row below the first owned row lives in the previous CTA
        csync<CS>();
        // ---- D6: w' -= G2 p --------------------------------------------------------
        {
          const T* pp = remote<CS>(pr, prev);
#pragma unroll
          for (int r = 0; r < RT; ++r) {
            const int jj = r * Cfg::G + grp, hr = jj + 2;
            const T pc = pr[jj * (2 * HSTR) + ci];
            const T pw = pr[jj * (2 * HSTR) + ((ci - 1) & MSK)];
            const T ps = jj > 0 ? pr[(jj - 1) * (2 * HSTR) + ci] : pp[(R - 1) * (2 * HSTR) + ci];
            wt[hr * N + ci] -= (pc - pw) * idx;
            wt[(HR + hr) * N + ci] -= (pc - ps) * idy;
          }
        }
        if (fused) {
          // u_n of the next step (and the row the previous CTA reads remotely)
          // before the arrive that lets the neighbours into the next stage
          if (stage == 3) {
            store_un();
            if (grp == 0) unrow0[ci] = wt[(HR + 2) * N + ci];
            tmem_wait_st();
          }
          __syncthreads();
          push_halos();
          cluster_arrive<CS>();
        }
      }
    }

    // ---- end of the time step: u_{n+1} becomes u_n -------------------------------
    if (!fused) {
      store_un();
      if (grp == 0) unrow0[ci] = wt[(HR + 2) * N + ci];
      tmem_wait_st();
    }
    if (a.save_every > 0 && a.traj != nullptr && (step % a.save_every) == 0) {
      const size_t tb = a.traj_batch > 0 ? (size_t)a.traj_batch : (size_t)gridDim.y;
      T* out = reinterpret_cast<T*>(a.traj) + ((size_t)snap * tb + traj) * 2 * NN;
#pragma unroll
      for (int r = 0; r < RT; ++r) {
        const int jj = r * Cfg::G + grp, hr = jj + 2;
        const size_t gi = (size_t)(row0 + jj) * N + ci;
        out[gi] = wt[hr * N + ci];
        out[NN + gi] = wt[(HR + hr) * N + ci];
      }
      ++snap;
    }
  }

#pragma unroll
  for (int r = 0; r < RT; ++r) {
    const int jj = r * Cfg::G + grp, hr = jj + 2;
    const size_t gi = (size_t)(row0 + jj) * N + ci;
    uout[gi] = wt[hr * N + ci];
    uout[NN + gi] = wt[(HR + hr) * N + ci];
  }
  // keep every CTA of the cluster resident until all DSMEM reads are done
  // (and, for the caller, every thread done with shared and tensor memory)
  if (fused) cluster_wait<CS>();  // the last stage's arrive
  tmem_fence_before_sync();
  csync<CS>();
  tmem_fence_after_sync();
}

template <typename T, int LOGN, int CS, int NT, int DORD>
__global__ void __launch_bounds__(NT, (FusedCfg<T, LOGN, CS, NT>::MIN_BLOCKS))
    fv_rollout_kernel(const FvArgs a) {
  using Cfg = FusedCfg<T, LOGN, CS, NT>;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint32_t* const tmem_slot = reinterpret_cast<uint32_t*>(smem + Cfg::OFF_TMEM);
  if ((threadIdx.x >> 5) == 0) tmem_alloc(tmem_slot, Cfg::TMEM_COLS);
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tmem_base = *tmem_slot;
  fv_rollout_body<T, LOGN, CS, NT, DORD>(a, (int)blockIdx.y, tmem_base);
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(tmem_base, Cfg::TMEM_COLS);
}

// ---------------------------------------------------------------------------
// Persistent rollout of a mixed batch: trajectories of different grid sizes
// (N = 16, 32, 64) and flow types, one CTA each, taken from a work list by the
// CTAs of one launch through an atomic counter until the list is exhausted
// (larger trajectories first, so the tail is short). Every trajectory runs the
// single-CTA configuration of the on-chip rollout at 256 threads, so its result
// is bit-identical to that of its own context's on-chip rollout.
// ---------------------------------------------------------------------------
struct MixedItem {
  FvArgs a;   // the trajectory's context arguments (u_in / u_out: its batch arrays)
  int traj;   // trajectory index in a.u_in / a.u_out
  int logn;   // 4, 5 or 6
};

constexpr int kMixedNT = 256;
constexpr int kMixedTmemCols = 128;  // the largest per-CTA need of N = 16 .. 64 at 256 threads
template <typename T>
constexpr size_t mixed_smem() {
  return cmax(FusedCfg<T, 4, 1, kMixedNT>::SMEM, cmax(FusedCfg<T, 5, 1, kMixedNT>::SMEM, FusedCfg<T, 6, 1, kMixedNT>::SMEM));
}
static_assert(FusedCfg<float, 6, 1, kMixedNT>::TMEM_COLS <= kMixedTmemCols &&
                  FusedCfg<float, 5, 1, kMixedNT>::TMEM_COLS <= kMixedTmemCols &&
                  FusedCfg<float, 4, 1, kMixedNT>::TMEM_COLS <= kMixedTmemCols,
              "tensor memory of the mixed rollout");

template <int DORD>
__global__ void __launch_bounds__(kMixedNT, 2)
    fv_mixed_rollout_kernel(const MixedItem* __restrict__ items, int n_items, unsigned* counter) {
  __shared__ uint32_t tslot;
  __shared__ int cur;
  if ((threadIdx.x >> 5) == 0) tmem_alloc(&tslot, kMixedTmemCols);
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tmem_base = tslot;
  for (;;) {
    if (threadIdx.x == 0) cur = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int i = cur;
    __syncthreads();  // every thread has read cur before thread 0 takes the next item
    if (i >= n_items) break;
    const FvArgs a = items[i].a;
    const int traj = items[i].traj;
    switch (items[i].logn) {
      case 4: fv_rollout_body<float, 4, 1, kMixedNT, DORD>(a, traj, tmem_base); break;
      case 5: fv_rollout_body<float, 5, 1, kMixedNT, DORD>(a, traj, tmem_base); break;
      default: fv_rollout_body<float, 6, 1, kMixedNT, DORD>(a, traj, tmem_base); break;
    }
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(tmem_base, kMixedTmemCols);
}

}  // namespace ldfv
