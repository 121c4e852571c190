// Mixed-precision ADER-DG predictor (Sec. 2.2 Eq. pde.nc.dg2) with the split
// final stage, laid out for the FP32 and FP64 pipes of one SM at once.
//
// A block of W warps takes W cells.  Phase A: each warp runs the FP32 Picard
// sweeps of its own cell (q <- u (x) 1 - Ktau x_tau sum_k c_k D x_k f_k(q)),
// synchronised by __syncwarp only; the last sweep yields the space-time
// correction dq = q - u, from which the warp writes trace(dq) (FP32) and the
// time-averaged flux changes sum_m w_m (F_k(u + dq_m) - F_k(u)) of its cell.
// Phase B: the block's threads share the FP64 terms of the W cells -- the
// fluxes F_k(u) at the spatial nodes, trace(u), and the volume part of the
// corrector u + sum_k c_k Mvol x_k fbar_k (Eq. pde.nc.gw2).  Blocks are
// persistent over groups of W cells, so blocks in phase A (FP32 pipe) and
// blocks in phase B (FP64 pipe) run side by side on every SM.
//
// The arithmetic of every output is that of the block-per-cell kernel
// (k_predictor, split branch); only the distribution of the work differs.
// With TC the sweeps' contractions run on the tensor pipe instead (mma.sync
// m16n8k8 TF32 with operands split into high and low TF32 parts, three
// products per tile: FP32-accurate).
#pragma once

#include "kernels_dg.cuh"

namespace adg {

// Per-cell shared memory of the warp-per-cell predictor, in floats:
//   uf  [NV ND]                   FP32 copy of u
//   qf  [max(NV NST, D NV ND)]    q, then S = sum_k c_k D x_k F_k, then the
//                                 time-averaged flux changes [D][NV][ND]
//   Ff  [D NV NST]                F_k(q); after the last sweep dq in
//                                 [0, NV NST) and fbar (FP64 [D][NV][ND])
//                                 behind it when it fits
// plus u (FP64 [NV ND]) and fbar when it does not fit in Ff.
template <int D, int N>
struct SplitLayout {
  using DM = Dims<D, N>;
  static constexpr int NV = DM::NV, ND = DM::ND, NST = DM::NST;
  // (float counts rounded up to even, so that every region starts 8-byte aligned)
  static constexpr int UF = (NV * ND + 1) / 2 * 2;
  static constexpr int QF = ((NV * NST > D * NV * ND) ? NV * NST : D * NV * ND) / 2 * 2 + 2;
  static constexpr int FF = D * NV * NST;
  static constexpr int FB_OFF = (NV * NST + 1) / 2 * 2;          // float offset of fbar in Ff
  // groups of time nodes of the flux-change sums (see k_predictor_split):
  // 3 or 2 when n divides evenly, the groups' partial sums fit in qf and the
  // ND nodes alone would leave most lanes of a round idle
  static constexpr int TSPLIT =
      (ND % 32 != 0 && ND < 64 && DM::n % 3 == 0 && 3 * D * NV * ND <= QF) ? 3
      : (ND % 32 != 0 && ND < 64 && DM::n % 2 == 0 && 2 * D * NV * ND <= QF) ? 2 : 1;
  static constexpr bool FB_IN_F = FB_OFF + 2 * D * NV * ND <= FF;
  // per cell: doubles (u, and fbar when it does not fit in Ff), then floats
  static constexpr int DBL = NV * ND + (FB_IN_F ? 0 : D * NV * ND);
  static constexpr int FLT = UF + QF + (FF + 1) / 2 * 2;
  static constexpr size_t cell_bytes = (size_t)DBL * 8 + (size_t)FLT * 4;
};

template <int D, int N, int W>
__host__ __device__ constexpr size_t split_smem_bytes() {
  using DM = Dims<D, N>;
  // operators: Mvol [n n], phi0, phi1 (FP64); phi0f, phi1f, wf (FP32)
  return (size_t)(DM::n * DM::n + 2 * DM::n) * 8 + (size_t)((3 * DM::n + 1) / 2 * 2) * 4 +
         (size_t)W * SplitLayout<D, N>::cell_bytes;
}

// Derivative phase of an FP32 sweep over one warp's cell, S = sum_k c_k D x_k
// F_k with the same operation order as picard_deriv_lines (which syncs the
// block between axes; here the warp).
template <int D, int N>
__device__ __forceinline__ void deriv_lines_warp(const float* __restrict__ F, float* __restrict__ S,
                                                 const float* c, int lane) {
  constexpr int n = N + 1, NV = D + 2, NST = ipow(n, D + 1), NL = NST / n;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const int st = (k == 0) ? 1 : (k == 1 ? n : n * n);
    const float ck = c[k];
    for (int e = lane; e < NV * NL; e += 32) {
      // line e of variable v = e / NL starts at v NST + (e % st) + ((e % NL) / st) st n,
      // which is n e - (n - 1)(e % st) (st divides NL and NST = n NL)
      const int base = n * e - (n - 1) * (e % st);
      const float* f = F + k * NV * NST + base;
      float x[n];
#pragma unroll
      for (int j = 0; j < n; ++j) x[j] = f[j * st];
      float* sl = S + base;
#pragma unroll
      for (int a = 0; a < n; ++a) {
        float acc = 0.0f;
#pragma unroll
        for (int j = 0; j < n; ++j) acc += c_Dmf[N][a * n + j] * x[j];
        if (k == 0) sl[a * st] = ck * acc;
        else sl[a * st] += ck * acc;
      }
    }
    if (k + 1 < D) __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Tensor-pipe contractions (TC): Y[line][a] = sum_j M[a][j] X[line][j] for
// 16 lines at a time with mma.sync.m16n8k8 (TF32 in, FP32 accumulate).  Each
// operand is split into a TF32 high part and the TF32 rounding of the rest,
// and hi*hi + lo*hi + hi*lo are accumulated (the lo*lo term is below FP32
// rounding), which keeps the contraction FP32-accurate.  n <= 8 nodes per
// line fill one k-step and one n-tile (padded with zeros); larger n use two.
// Fragment layout of m16n8k8 (row-major A 16x8, column-major B 8x8,
// C 16x8), thread lane = 4 g + t: a0 = A[g][t], a1 = A[g+8][t],
// a2 = A[g][t+4], a3 = A[g+8][t+4]; b0 = B[t][g], b1 = B[t+4][g];
// c0 = C[g][2t], c1 = C[g][2t+1], c2 = C[g+8][2t], c3 = C[g+8][2t+1].
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t tf32_of(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Split x into its TF32 high part and the TF32 rounding of the remainder.
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_of(x);
  lo = tf32_of(x - __uint_as_float(hi));
}

// B fragments (high, low) of the operator M (n x n, row a = output node,
// column j = input node) for k-step ks and n-tile nt: B[j][a] = M[a][j].
template <int n>
__device__ __forceinline__ void op_fragments(const float* M, int ks, int nt, int lane, uint32_t* bh,
                                             uint32_t* bl) {
  const int g = lane >> 2, t = lane & 3;
  const int a = nt * 8 + g;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int j = ks * 8 + t + 4 * r;
    const float x = (a < n && j < n) ? M[a * n + j] : 0.0f;
    split_tf32(x, bh[r], bl[r]);
  }
}

// The lines of one contraction: line L (0 <= L < nlines) starts at float
// offset base(L) of the source with stride `st` between its n nodes; the
// result goes to the same offsets of the destination.  `Line` maps a line
// index to its base offset.  Mode 0: dst = scale * Y; mode 1: dst += scale *
// Y; mode 2: dst = u(line) - Y with u given per line by `ubase`.
template <int n, int MODE, typename Line, typename UOf>
__device__ __forceinline__ void contract_tc(const float* src, float* dst, int nlines, int st,
                                            Line base, float scale, UOf uof,
                                            const uint32_t (*bh)[2], const uint32_t (*bl)[2],
                                            int lane) {
  constexpr int KS = (n + 7) / 8;      // k-steps
  constexpr int NT = (n + 7) / 8;      // n-tiles
  const int g = lane >> 2, t = lane & 3;
  for (int L0 = 0; L0 < nlines; L0 += 16) {
    const int La = L0 + g, Lb = L0 + g + 8;
    const bool va = La < nlines, vb = Lb < nlines;
    const int oa = va ? base(La) : 0, ob = vb ? base(Lb) : 0;
    float acc[NT][4];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[nt][r] = 0.0f;
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      uint32_t ah[4], al[4];
      const int j0 = ks * 8 + t, j1 = ks * 8 + t + 4;
      split_tf32((va && j0 < n) ? src[oa + j0 * st] : 0.0f, ah[0], al[0]);
      split_tf32((vb && j0 < n) ? src[ob + j0 * st] : 0.0f, ah[1], al[1]);
      split_tf32((va && j1 < n) ? src[oa + j1 * st] : 0.0f, ah[2], al[2]);
      split_tf32((vb && j1 < n) ? src[ob + j1 * st] : 0.0f, ah[3], al[3]);
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        mma_tf32(acc[nt], al, bh[ks * NT + nt]);
        mma_tf32(acc[nt], ah, bl[ks * NT + nt]);
        mma_tf32(acc[nt], ah, bh[ks * NT + nt]);
      }
    }
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int a = nt * 8 + 2 * t + (r & 1);
        const bool row_ok = (r < 2) ? va : vb;
        if (a < n && row_ok) {
          const int o = ((r < 2) ? oa : ob) + a * st;
          const float y = acc[nt][r];
          if (MODE == 0) dst[o] = scale * y;
          else if (MODE == 1) dst[o] += scale * y;
          else dst[o] = uof((r < 2) ? La : Lb, a) - y;
        }
      }
  }
}

// One warp's FP32 Picard sweep contractions on the tensor pipe: S = sum_k c_k
// D x_k F_k (into qf), then q = u - Ktau x_tau S (or dq = -Ktau x_tau S).
template <int D, int N>
struct TcSweep {
  static constexpr int n = N + 1, NV = D + 2, ND = ipow(n, D), NST = ipow(n, D + 1);
  static constexpr int KS = (n + 7) / 8, NT = (n + 7) / 8;
  // B fragments (high and low TF32 parts) of D and Ktau per (k-step, n-tile)
  uint32_t dh[KS * NT][2], dl[KS * NT][2];
  uint32_t kh[KS * NT][2], kl[KS * NT][2];

  __device__ __forceinline__ void load(int lane) {
#pragma unroll
    for (int ks = 0; ks < KS; ++ks)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        op_fragments<n>(c_Dmf[N], ks, nt, lane, dh[ks * NT + nt], dl[ks * NT + nt]);
        op_fragments<n>(c_Ktf[N], ks, nt, lane, kh[ks * NT + nt], kl[ks * NT + nt]);
      }
  }

  // derivative phase: the lines along axis k of every variable
  __device__ __forceinline__ void deriv(const float* F, float* S, const float* c, int lane) const {
    constexpr int NL = NST / n;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const int st = (k == 0) ? 1 : (k == 1 ? n : n * n);
      // line L = v NL + r starts at v NST + r % st + (r / st) st n
      auto base = [st](int L) {
        const int v = L / NL, r = L - v * NL;
        return v * NST + r % st + (r / st) * (st * n);
      };
      auto nou = [](int, int) { return 0.0f; };
      if (k == 0)
        contract_tc<n, 0>(F, S, NV * NL, st, base, c[0], nou, dh, dl, lane);
      else
        contract_tc<n, 1>(F + k * NV * NST, S, NV * NL, st, base, c[k], nou, dh, dl, lane);
      if (k + 1 < D) __syncwarp();
    }
  }

  // time phase: out = u - Ktau S along tau (lines: variable and spatial node);
  // u == nullptr gives dq = -Ktau S
  __device__ __forceinline__ void time(const float* S, float* out, const float* u, int lane) const {
    auto base = [](int L) {
      const int v = L / ND, i = L - v * ND;
      return v * NST + i;
    };
    auto uof = [u](int L, int) { return u ? u[L] : 0.0f; };
    contract_tc<n, 2>(S, out, NV * ND, ND, base, 1.0f, uof, kh, kl, lane);
  }
};

template <int D, int N, int W, bool TC>
__global__ void __launch_bounds__(32 * W) k_predictor_split(Batch bt) {
  using DM = Dims<D, N>;
  using LY = SplitLayout<D, N>;
  constexpr int n = DM::n, NV = DM::NV, ND = DM::ND, NST = DM::NST, NF = DM::NF, NT = DM::NT;
  extern __shared__ double sm[];
  double* Mv = sm;
  double* ph0 = Mv + n * n;
  double* ph1 = ph0 + n;
  float* ph0f = reinterpret_cast<float*>(ph1 + n);
  float* ph1f = ph0f + n;
  float* wf = ph1f + n;
  unsigned char* cells0 = reinterpret_cast<unsigned char*>(ph0f + (3 * n + 1) / 2 * 2);
  __shared__ const Params* s_pp[W];
  __shared__ long long s_cell[W];
  __shared__ int s_on[W];

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const Ops* o = bt.pps[0]->ops;      // every state of a batch has degree N
  for (int i = tid; i < n * n; i += 32 * W) Mv[i] = o->Mvol[i];
  for (int i = tid; i < n; i += 32 * W) {
    ph0[i] = o->phi0[i];
    ph1[i] = o->phi1[i];
    ph0f[i] = (float)o->phi0[i];
    ph1f[i] = (float)o->phi1[i];
    wf[i] = (float)o->w[i];
  }
  // this warp's cell storage
  unsigned char* mine = cells0 + (size_t)w * LY::cell_bytes;
  double* u = reinterpret_cast<double*>(mine);
  float* uf = reinterpret_cast<float*>(u + LY::DBL);
  float* qf = uf + LY::UF;
  float* Ff = qf + LY::QF;
  TcSweep<D, N> tc;
  if constexpr (TC) tc.load(lane);
  __syncthreads();

  const long long total = bt.pre[bt.n];
  const long long ngroups = (total + W - 1) / W;
  for (long long grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    // ---- phase A: FP32 sweeps of this warp's cell ----
    const long long g = grp * W + w;
    bool on = false;
    const Params* pp = nullptr;
    long long cell = 0;
    if (g < total) {
      const int sidx = batch_state(bt, g);
      pp = bt.pps[sidx];
      cell = g - bt.pre[sidx];
      on = *pp->b.dt > 0.0;         // state idle this step otherwise
    }
    if (lane == 0) {
      s_pp[w] = pp;
      s_cell[w] = cell;
      s_on[w] = on ? 1 : 0;
      // the DOF block of the cell this warp takes next, into L2 while this one runs
      constexpr unsigned UBYTES = NV * ND * sizeof(double);
      const long long gn = g + (long long)gridDim.x * W;
      if (UBYTES % 16 == 0 && gn < total) {
        const int sn = batch_state(bt, gn);
        const Params* pn = bt.pps[sn];
        bulk_prefetch_l2(pn->b.U[pn->cur] + (gn - bt.pre[sn]) * (NV * ND), UBYTES);
      }
    }
    if (on) {
      const Params& p = *pp;
      float cf[3];
#pragma unroll
      for (int k = 0; k < D; ++k) cf[k] = (float)p.b.coef[k];
      const float gm1f = (float)(p.gamma - 1.0);
      const double* Uc = p.b.U[p.cur] + cell * (NV * ND);
      for (int e = lane; e < NV * ND; e += 32) {
        const double x = Uc[e];
        u[e] = x;
        uf[e] = (float)x;
      }
      __syncwarp();
      const int n32 = p.iters;           // all sweeps in FP32 (split final stage)
      // The first sweep starts from q^0 = u (x) 1, whose fluxes and their
      // derivatives S are the same at every time node: both phases run on the
      // n^d spatial nodes only (time slice 0), and q^1_m = u - kappa_m S with
      // kappa_m = sum_j Ktau[m][j] (dq = -kappa_m S when it is also the last).
      for (int i = lane; i < ND; i += 32) {
        float Q[NV], Fl[D][D + 2];
#pragma unroll
        for (int v = 0; v < NV; ++v) Q[v] = uf[v * ND + i];
        euler_fluxes<D, float>(Q, gm1f, Fl);
#pragma unroll
        for (int k = 0; k < D; ++k)
#pragma unroll
          for (int v = 0; v < NV; ++v) Ff[(k * NV + v) * NST + i] = Fl[k][v];
      }
      __syncwarp();
#pragma unroll
      for (int k = 0; k < D; ++k) {
        constexpr int NLS = ND / n;        // lines of one variable's time slice along an axis
        const int st = (k == 0) ? 1 : (k == 1 ? n : n * n);
        const float ck = cf[k];
        for (int e = lane; e < NV * NLS; e += 32) {
          const int v = e / NLS, r = e - v * NLS;
          const int base = v * NST + n * r - (n - 1) * (r % st);
          float x[n];
#pragma unroll
          for (int j = 0; j < n; ++j) x[j] = Ff[k * NV * NST + base + j * st];
#pragma unroll
          for (int a = 0; a < n; ++a) {
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < n; ++j) acc += c_Dmf[N][a * n + j] * x[j];
            if (k == 0) qf[base + a * st] = ck * acc;
            else qf[base + a * st] += ck * acc;
          }
        }
        __syncwarp();
      }
      {
        float kap[n];
#pragma unroll
        for (int m = 0; m < n; ++m) {
          float t = 0.0f;
#pragma unroll
          for (int j = 0; j < n; ++j) t += c_Ktf[N][m * n + j];
          kap[m] = t;
        }
        float* out = n32 == 1 ? Ff : qf;
        for (int e = lane; e < NV * ND; e += 32) {
          const int v = e / ND, i = e - v * ND;
          const float sv = qf[v * NST + i];
          const float u0 = n32 == 1 ? 0.0f : uf[e];
#pragma unroll
          for (int m = 0; m < n; ++m) out[v * NST + i + m * ND] = u0 - kap[m] * sv;
        }
      }
      __syncwarp();
      for (int it = 1; it < n32; ++it) {
        picard_flux<D, n, float>(qf, Ff, gm1f, lane, 32);
        __syncwarp();
        if constexpr (TC) tc.deriv(Ff, qf, cf, lane);
        else deriv_lines_warp<D, N>(Ff, qf, cf, lane);
        __syncwarp();
        if (it == n32 - 1) {
          // the last sweep: dq = -Ktau S into Ff
          if constexpr (TC) tc.time(qf, Ff, nullptr, lane);
          else picard_time_dq<D, N>(qf, Ff, lane, 32);
        } else {
          if constexpr (TC) tc.time(qf, qf, uf, lane);
          else picard_time_cf<D, N>(qf, uf, lane, 32);
        }
        __syncwarp();
      }
      const float* dq = Ff;
      // trace(dq) in FP32 (the split trace layout of k_predictor: per cell,
      // axis k and side s a block of NV NT doubles, trace(u) [NV][NF] in FP64
      // then trace(dq) [NV][NT] in FP32), by lines: the n nodes of each line
      // along axis k give the traces on both faces normal to k, and the line's
      // index r within its variable is the trace's index ts + NF m
      double* tr = p.b.trace + cell * (size_t)(D * 2 * NV * NT);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        constexpr int NL = NST / n;
        const int st = (k == 0) ? 1 : (k == 1 ? n : n * n);
        float* t0 = reinterpret_cast<float*>(tr + (2 * k) * (NV * NT) + NV * NF);
        float* t1 = reinterpret_cast<float*>(tr + (2 * k + 1) * (NV * NT) + NV * NF);
        static_assert(NL == NT, "a variable has as many lines along an axis as trace values per side");
        for (int e = lane; e < NV * NL; e += 32) {
          const float* d = dq + n * e - (n - 1) * (e % st);
          float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
          for (int a = 0; a < n; ++a) {
            a0 += ph0f[a] * d[a * st];
            a1 += ph1f[a] * d[a * st];
          }
          t0[e] = a0;     // [v][ts + NF m] with v NT + ts + NF m = e
          t1[e] = a1;
        }
      }
      // time-averaged flux changes per spatial node, into qf: the products
      // w_m G rounded and summed over the time nodes in order.  When a warp
      // has few nodes (ND not much larger than 32 or far below it) the time
      // nodes are split in TS groups, each lane summing one group of one node,
      // and the groups' partial sums are added in group order afterwards.
      constexpr int TS = LY::TSPLIT, MG = n / TS;
      float* dFb = qf;
      for (int t = lane; t < ND * TS; t += 32) {
        const int i = t % ND, grp = t / ND;
        float U[NV], acc[D][D + 2];
#pragma unroll
        for (int v = 0; v < NV; ++v) U[v] = uf[v * ND + i];
#pragma unroll
        for (int k = 0; k < D; ++k)
#pragma unroll
          for (int v = 0; v < NV; ++v) acc[k][v] = 0.0f;
        for (int mm = 0; mm < MG; ++mm) {
          const int m = grp * MG + mm;
          float dQ[NV], G[D][D + 2];
#pragma unroll
          for (int v = 0; v < NV; ++v) dQ[v] = dq[v * NST + i + m * ND];
          euler_flux_delta<D>(U, dQ, gm1f, G);
          const float wm = wf[m];
#pragma unroll
          for (int k = 0; k < D; ++k)
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[k][v] = __fadd_rn(acc[k][v], __fmul_rn(wm, G[k][v]));
        }
#pragma unroll
        for (int k = 0; k < D; ++k)
#pragma unroll
          for (int v = 0; v < NV; ++v) dFb[(grp * D * NV + k * NV + v) * ND + i] = acc[k][v];
      }
      if constexpr (TS > 1) {
        __syncwarp();
        for (int e = lane; e < D * NV * ND; e += 32) {
          float x = dFb[e];
#pragma unroll
          for (int grp = 1; grp < TS; ++grp) x = __fadd_rn(x, dFb[grp * D * NV * ND + e]);
          dFb[e] = x;
        }
      }
    }
    __syncthreads();

    // ---- phase B: FP64 terms of the block's W cells ----
    // B1: fbar_k = F_k(u) + the FP32 flux changes at the spatial nodes
    for (int t = tid; t < W * ND; t += 32 * W) {
      const int ww = t / ND, i = t - ww * ND;
      if (!s_on[ww]) continue;
      const Params& p = *s_pp[ww];
      unsigned char* cb = cells0 + (size_t)ww * LY::cell_bytes;
      const double* uu = reinterpret_cast<const double*>(cb);
      const float* dF = reinterpret_cast<const float*>(uu + LY::DBL) + LY::UF;
      double* fb = LY::FB_IN_F ? reinterpret_cast<double*>(const_cast<float*>(dF) + LY::QF + LY::FB_OFF)
                               : const_cast<double*>(uu) + NV * ND;
      double Q[NV], Fl[D][D + 2];
#pragma unroll
      for (int v = 0; v < NV; ++v) Q[v] = uu[v * ND + i];
      euler_fluxes<D, double>(Q, p.gamma - 1.0, Fl);
#pragma unroll
      for (int k = 0; k < D; ++k)
#pragma unroll
        for (int v = 0; v < NV; ++v)
          fb[(k * NV + v) * ND + i] = Fl[k][v] + widen_f32(dF[(k * NV + v) * ND + i]);
    }
    // trace(u) in FP64 (the split layout's [NV][NF] part), by lines of n
    // spatial nodes along axis k: both faces normal to k from one line
    for (int t = tid; t < W * D * NV * NF; t += 32 * W) {
      const int ww = t / (D * NV * NF);
      int e = t - ww * (D * NV * NF);
      if (!s_on[ww]) continue;
      const int k = e / (NV * NF);
      e -= k * (NV * NF);
      const int v = e / NF, r = e - v * NF;
      const int st = (k == 0) ? 1 : (k == 1 ? n : n * n);
      const Params& p = *s_pp[ww];
      const double* uu = reinterpret_cast<const double*>(cells0 + (size_t)ww * LY::cell_bytes) +
                         v * ND + r % st + (r / st) * (st * n);
      double a0 = 0.0, a1 = 0.0;
#pragma unroll
      for (int a = 0; a < n; ++a) {
        a0 += ph0[a] * uu[a * st];
        a1 += ph1[a] * uu[a * st];
      }
      double* tr = p.b.trace + s_cell[ww] * (size_t)(D * 2 * NV * NT);
      tr[(2 * k) * (NV * NT) + v * NF + r] = a0;
      tr[(2 * k + 1) * (NV * NT) + v * NF + r] = a1;
    }
    __syncthreads();
    // B2: the volume part of the candidate, u + sum_k c_k Mvol x_k fbar_k
    for (int t = tid; t < W * NV * ND; t += 32 * W) {
      const int ww = t / (NV * ND), e = t - ww * (NV * ND);
      if (!s_on[ww]) continue;
      const Params& p = *s_pp[ww];
      unsigned char* cb = cells0 + (size_t)ww * LY::cell_bytes;
      const double* uu = reinterpret_cast<const double*>(cb);
      const float* dF = reinterpret_cast<const float*>(uu + LY::DBL) + LY::UF;
      const double* fb = LY::FB_IN_F
                             ? reinterpret_cast<const double*>(dF + LY::QF + LY::FB_OFF)
                             : uu + NV * ND;
      const int v = e / ND, i = e - v * ND;
      double acc = uu[e];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const int st = (k == 0) ? 1 : (k == 1 ? n : n * n);
        const int ak = (i / st) % n;
        const double* f = fb + (k * NV + v) * ND + (i - ak * st);
        double tt = 0.0;
#pragma unroll
        for (int j = 0; j < n; ++j) tt += Mv[ak * n + j] * f[j * st];
        acc += p.b.coef[k] * tt;
      }
      p.b.U[1 - p.cur][s_cell[ww] * (NV * ND) + e] = acc;
    }
    __syncthreads();
  }
}

}  // namespace adg
