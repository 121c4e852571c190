// ADER-DG kernels: space-time predictor (Sec. 2.2 Eq. pde.nc.dg2), DG face
// fluxes and corrector (Sec. 2.3 Eq. pde.nc.gw2) fused with the a-posteriori
// detector (Sec. 4.3 Eqs. positivity, dmp, relax).
#pragma once

#include <climits>

#include "adg_internal.h"

namespace adg {

template <int D, int N>
struct Dims {
  static constexpr int n = N + 1;
  static constexpr int NV = D + 2;
  static constexpr int ND = ipow(n, D);          // spatial nodes per cell
  static constexpr int NST = ipow(n, D + 1);     // space-time nodes per cell
  static constexpr int NF = ipow(n, D - 1);      // tangential nodes per face
  static constexpr int NT = NF * n;              // tangential x time nodes per face
  static constexpr int Ns = 2 * N + 1;
  static constexpr int NSD = ipow(Ns, D);        // subcells per cell
  static constexpr int NSF = ipow(Ns, D - 1);    // sub-faces per cell face
  static constexpr int L = Ns + 6;               // limiter patch width (3 ghost layers)
  static constexpr int LD = ipow(L, D);
  static constexpr int NE = Ns + 2;              // reconstructed block -1..Ns
  static constexpr int NED = ipow(NE, D);
  static constexpr int NST3 = ipow(3, D + 1);    // subcell space-time nodes
  static constexpr int ND3 = ipow(3, D);
};

// Predictor block shape.  The mixed kernel at high 2D degrees is latency
// bound with one 128-thread block per SM (measured: 4 warps per SM, FP64 pipe
// 41% busy at N = 9); 256 threads capped at 128 registers, two blocks per SM,
// hide the FP32 and FP64 latencies.  Below N = 6 the 2D mixed kernel runs 128
// threads capped at 102 registers, five blocks per SM (measured against four
// blocks at N = 4 and 5: 8% and 4% faster; 160 threads: 17% slower at N = 4;
// 256 threads: 40% slower), the 3D mixed kernel 160 threads, four blocks per
// SM (9% faster than 128 at N = 3).  The FP64 kernel keeps the FP64 pipe busy
// as it is and runs faster without the register cap.
template <int D, int N, bool MIXED>
struct PredShape {
  static constexpr bool wide = MIXED && D == 2 && N >= 6;
  static constexpr bool narrow3 = MIXED && D == 3;
  static constexpr int threads = wide ? 256 : (narrow3 ? 160 : 128);   // launched per block
  static constexpr int bound = (MIXED && !wide) ? threads : 256;       // __launch_bounds__ maximum
  // registers: <= 102 for the narrow mixed kernels (five 128- or four
  // 160-thread blocks per SM), <= 128 otherwise (two 256-thread or four
  // 128-thread blocks), except the FP64 kernel at 2D N >= 6, which would spill
  // under that cap
  static constexpr int min_blocks =
      narrow3 ? 4 : ((MIXED && !wide) ? 5 : ((!MIXED && D == 2 && N >= 6) ? 1 : 2));
};

// ---------------------------------------------------------------------------
// Picard phases on one space-time block of n^(D+1) nodes (Eq. pde.nc.dg2):
//   q <- u (x) 1 - Ktau x_tau sum_k c_k D x_k f_k(q),  c_k = dt / dx_k.
// Work items are spread over threads tid .. (step nth).
// ---------------------------------------------------------------------------
template <int D, int n, typename T>
__device__ __forceinline__ void picard_flux(const T* __restrict__ q, T* __restrict__ F, T gm1,
                                            int tid, int nth) {
  constexpr int NV = D + 2, NST = ipow(n, D + 1);
  for (int l = tid; l < NST; l += nth) {
    T Q[NV];
    T Fl[D][D + 2];
#pragma unroll
    for (int v = 0; v < NV; ++v) Q[v] = q[v * NST + l];
    euler_fluxes<D, T>(Q, gm1, Fl);
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
      for (int v = 0; v < NV; ++v) F[(k * NV + v) * NST + l] = Fl[k][v];
  }
}

template <int D, int n, typename T>
__device__ __forceinline__ void picard_deriv(const T* __restrict__ F, T* __restrict__ S,
                                             const T* __restrict__ Dm, const T* c, int tid,
                                             int nth) {
  constexpr int NV = D + 2, NST = ipow(n, D + 1);
  for (int e = tid; e < NV * NST; e += nth) {
    const int v = e / NST, l = e - v * NST;
    T s = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const int st = (k == 0) ? 1 : (k == 1 ? n : n * n);
      const int ak = (l / st) % n;
      const T* f = F + (k * NV + v) * NST + (l - ak * st);
      const T* dr = Dm + ak * n;
      T acc = T(0);
#pragma unroll
      for (int j = 0; j < n; ++j) acc += dr[j] * f[j * st];
      s += c[k] * acc;
    }
    S[e] = s;
  }
}

template <int D, int n, typename T, typename UT>
__device__ __forceinline__ void picard_time(T* __restrict__ q, const UT* __restrict__ u,
                                            const T* __restrict__ Kt, int tid, int nth) {
  constexpr int NV = D + 2, ND = ipow(n, D), NST = ipow(n, D + 1);
  for (int e = tid; e < NV * ND; e += nth) {
    const int v = e / ND, i = e - v * ND;
    T Sl[n];
#pragma unroll
    for (int m = 0; m < n; ++m) Sl[m] = q[v * NST + i + m * ND];
    const T u0 = (T)u[v * ND + i];
#pragma unroll
    for (int m = 0; m < n; ++m) {
      T acc = T(0);
#pragma unroll
      for (int j = 0; j < n; ++j) acc += Kt[m * n + j] * Sl[j];
      q[v * NST + i + m * ND] = u0 - acc;
    }
  }
}

// FP32 Picard operators D and Ktau of every degree N (index N) in constant
// memory, one copy per translation unit (filled by upload_picard_constants):
// with the loops unrolled every operator entry is a constant-bank operand of
// its FMA, so the FP32 sweeps load only their data from shared memory.
static __constant__ float c_Dmf[MAXN][MAXN * MAXN];
static __constant__ float c_Ktf[MAXN][MAXN * MAXN];
// the degree-2 subcell predictor's operators (3 nodes), likewise
static __constant__ float c_D3f[9];
static __constant__ float c_K3f[9];

// Derivative and time phases of an FP32 sweep of the subcell predictor with
// its operators from constant memory; one output per work item and no
// barrier inside (the caller's thread groups run them under a condition).
// Operation order as in picard_deriv / picard_time.
template <int D>
__device__ __forceinline__ void picard_deriv_sub(const float* __restrict__ F, float* __restrict__ S,
                                                 const float* c, int tid, int nth) {
  constexpr int n = 3, NV = D + 2, NST = ipow(n, D + 1);
  for (int e = tid; e < NV * NST; e += nth) {
    const int v = e / NST, l = e - v * NST;
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const int st = (k == 0) ? 1 : (k == 1 ? n : n * n);
      const int ak = (l / st) % n;
      const float* f = F + (k * NV + v) * NST + (l - ak * st);
      float x[n];
#pragma unroll
      for (int j = 0; j < n; ++j) x[j] = f[j * st];
      // row ak of D3 from constant memory (ak is 0, 1 or 2)
      const float d0 = ak == 0 ? c_D3f[0] : (ak == 1 ? c_D3f[3] : c_D3f[6]);
      const float d1 = ak == 0 ? c_D3f[1] : (ak == 1 ? c_D3f[4] : c_D3f[7]);
      const float d2 = ak == 0 ? c_D3f[2] : (ak == 1 ? c_D3f[5] : c_D3f[8]);
      float acc = 0.0f;
      acc += d0 * x[0];
      acc += d1 * x[1];
      acc += d2 * x[2];
      s += c[k] * acc;
    }
    S[e] = s;
  }
}

template <int D>
__device__ __forceinline__ void picard_time_sub(float* __restrict__ q, const float* __restrict__ u,
                                                int tid, int nth) {
  constexpr int n = 3, NV = D + 2, ND = ipow(n, D), NST = ipow(n, D + 1);
  for (int e = tid; e < NV * ND; e += nth) {
    const int v = e / ND, i = e - v * ND;
    float Sl[n];
#pragma unroll
    for (int m = 0; m < n; ++m) Sl[m] = q[v * NST + i + m * ND];
    const float u0 = u[v * ND + i];
#pragma unroll
    for (int m = 0; m < n; ++m) {
      float acc = 0.0f;
#pragma unroll
      for (int j = 0; j < n; ++j) acc += c_K3f[m * n + j] * Sl[j];
      q[v * NST + i + m * ND] = u0 - acc;
    }
  }
}

// Derivative phase of an FP32 sweep, S = sum_k c_k D x_k F_k, one thread per
// line of n nodes along axis k: the line's n fluxes are loaded once and give
// n outputs (n independent FMA chains).  The axes run one after the other
// (S is written for k = 0 and accumulated after), with the same operation
// order per output as picard_deriv.
template <int D, int N>
__device__ __forceinline__ void picard_deriv_lines(const float* __restrict__ F, float* __restrict__ S,
                                                   const float* c, int tid, int nth) {
  constexpr int n = N + 1, NV = D + 2, NST = ipow(n, D + 1), NL = NST / n;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const int st = (k == 0) ? 1 : (k == 1 ? n : n * n);
    const float ck = c[k];
    for (int e = tid; e < NV * NL; e += nth) {
      const int v = e / NL, r = e - v * NL;
      const int base = r % st + (r / st) * (st * n);
      const float* f = F + (k * NV + v) * NST + base;
      float x[n];
#pragma unroll
      for (int j = 0; j < n; ++j) x[j] = f[j * st];
      float* sl = S + v * NST + base;
#pragma unroll
      for (int a = 0; a < n; ++a) {
        float acc = 0.0f;
#pragma unroll
        for (int j = 0; j < n; ++j) acc += c_Dmf[N][a * n + j] * x[j];
        if (k == 0) sl[a * st] = ck * acc;
        else sl[a * st] += ck * acc;
      }
    }
    if (k + 1 < D) __syncthreads();
  }
}

// Time phase of an FP32 sweep, q <- u - Ktau S, with Ktau from constant memory.
template <int D, int N>
__device__ __forceinline__ void picard_time_cf(float* __restrict__ q, const float* __restrict__ u,
                                               int tid, int nth) {
  constexpr int n = N + 1, NV = D + 2, ND = ipow(n, D), NST = ipow(n, D + 1);
  for (int e = tid; e < NV * ND; e += nth) {
    const int v = e / ND, i = e - v * ND;
    float Sl[n];
#pragma unroll
    for (int m = 0; m < n; ++m) Sl[m] = q[v * NST + i + m * ND];
    const float u0 = u[v * ND + i];
#pragma unroll
    for (int m = 0; m < n; ++m) {
      float acc = 0.0f;
#pragma unroll
      for (int j = 0; j < n; ++j) acc += c_Ktf[N][m * n + j] * Sl[j];
      q[v * NST + i + m * ND] = u0 - acc;
    }
  }
}

// The time phase of the last FP32 Picard sweep when no FP64 sweep follows:
// only the space-time correction dq = q - u = -Ktau S is formed (FP32, from
// the sweep's S = sum_k c_k D x_k f_k(q)); the final stage adds it to the
// FP64 u term by term (face traces, fluxes), so q carries no FP32 rounding of
// u itself (the dominant error of a plain FP32 sweep).
template <int D, int N>
__device__ __forceinline__ void picard_time_dq(const float* __restrict__ S,
                                               float* __restrict__ dq, int tid, int nth) {
  constexpr int n = N + 1, NV = D + 2, ND = ipow(n, D), NST = ipow(n, D + 1);
  for (int e = tid; e < NV * ND; e += nth) {
    const int v = e / ND, i = e - v * ND;
    float Sl[n];
#pragma unroll
    for (int m = 0; m < n; ++m) Sl[m] = S[v * NST + i + m * ND];
#pragma unroll
    for (int m = 0; m < n; ++m) {
      float acc = 0.0f;
#pragma unroll
      for (int j = 0; j < n; ++j) acc += c_Ktf[N][m * n + j] * Sl[j];
      dq[v * NST + i + m * ND] = -acc;
    }
  }
}

// Euler flux difference F_k(U + dQ) - F_k(U), k = 0..D-1, in FP32 and in a
// form where every term carries a factor of dQ (velocity change
// dv = (dm - v drho) / (rho + drho), pressure change
// dp = (gamma - 1)(dE - d(m.v)/2) with d(m.v) = sum_j dm_j (v_j + dv_j) + m_j dv_j),
// so its rounding error is relative to the change, not to the flux: with
// F(U) in FP64 the sum equals F(U + dQ) to FP32 rounding of the correction.
template <int D>
__device__ __forceinline__ void euler_flux_delta(const float* U, const float* dQ, float gm1,
                                                 float (*G)[D + 2]) {
  const float r = 1.0f / U[0];
  const float r1 = 1.0f / (U[0] + dQ[0]);
  float v[D], dv[D];
  float mv = 0.0f, dmv = 0.0f;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    v[j] = U[1 + j] * r;
    mv += U[1 + j] * v[j];
    dv[j] = (dQ[1 + j] - v[j] * dQ[0]) * r1;
  }
#pragma unroll
  for (int j = 0; j < D; ++j) dmv += dQ[1 + j] * (v[j] + dv[j]) + U[1 + j] * dv[j];
  const float Ep = U[D + 1] + gm1 * (U[D + 1] - 0.5f * mv);
  const float dp = gm1 * (dQ[D + 1] - 0.5f * dmv);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const float vk1 = v[k] + dv[k];
    G[k][0] = dQ[1 + k];
#pragma unroll
    for (int j = 0; j < D; ++j) G[k][1 + j] = dQ[1 + j] * vk1 + U[1 + j] * dv[k];
    G[k][1 + k] += dp;
    G[k][D + 1] = (dQ[D + 1] + dp) * vk1 + Ep * dv[k];
  }
}

// Apply a matrix along axis k of a (nv, e0, e1, e2) tensor (x fastest):
// out[v][.., r, ..] = sum_c M[r * cols + c] in[v][.., c, ..].
// ein: extents of `in`; out has extent `rows` along k.
template <int D>
__device__ __forceinline__ void apply_axis(const double* __restrict__ in, double* __restrict__ out,
                                           const double* __restrict__ M, int rows, int cols, int k,
                                           const int* ein, int nv, int tid, int nth) {
  int eout[3] = {1, 1, 1};
  int insz = 1, outsz = 1;
  for (int j = 0; j < D; ++j) {
    eout[j] = (j == k) ? rows : ein[j];
    insz *= ein[j];
    outsz *= eout[j];
  }
  int stride = 1;
  for (int j = 0; j < k; ++j) stride *= ein[j];
  for (int e = tid; e < nv * outsz; e += nth) {
    const int v = e / outsz;
    int r = e - v * outsz;
    int idx[3] = {0, 0, 0};
    for (int j = 0; j < D; ++j) {
      idx[j] = r % eout[j];
      r /= eout[j];
    }
    int off = 0, s = 1;
    for (int j = 0; j < D; ++j) {
      off += (j == k ? 0 : idx[j]) * s;
      s *= ein[j];
    }
    const double* src = in + v * insz + off;
    const double* mr = M + idx[k] * cols;
    double acc = 0.0;
    for (int c = 0; c < cols; ++c) acc += mr[c] * src[c * stride];
    out[e] = acc;
  }
}

// Tensor projection / reconstruction of all variables of one cell through two
// buffers: NV variables, NI -> NO points per axis, matrix M[NO][NI]; every
// index division is by a constant.
template <int D, int NV, int NI, int NO, int K, typename T = double>
__device__ __forceinline__ void apply_pass_ct(const T* __restrict__ in, T* __restrict__ out,
                                              const T* __restrict__ M, int tid, int nth) {
  constexpr int I0 = (0 < K) ? NO : NI, I1 = (1 < K) ? NO : NI, I2 = (2 < K) ? NO : NI;
  constexpr int O0 = (0 <= K) ? NO : NI, O1 = (1 <= K) ? NO : NI, O2 = (2 <= K) ? NO : NI;
  constexpr int E1 = (D > 1) ? 1 : 0, E2 = (D > 2) ? 1 : 0;
  constexpr int ISZ = I0 * (E1 ? I1 : 1) * (E2 ? I2 : 1);
  constexpr int OSZ = O0 * (E1 ? O1 : 1) * (E2 ? O2 : 1);
  constexpr int STRIDE = (K == 0) ? 1 : (K == 1 ? I0 : I0 * I1);
  for (int e = tid; e < NV * OSZ; e += nth) {
    const int v = e / OSZ;
    int r = e - v * OSZ;
    const int x0 = r % O0;
    r /= O0;
    const int x1 = E1 ? r % O1 : 0;
    const int x2 = E2 ? r / O1 : 0;
    const int xk = (K == 0) ? x0 : (K == 1 ? x1 : x2);
    const int off = (K == 0 ? 0 : x0) + I0 * ((K == 1 ? 0 : x1) + I1 * (K == 2 ? 0 : x2));
    const T* src = in + v * ISZ + off;
    const T* mr = M + xk * NI;
    T acc = T(0);
#pragma unroll
    for (int c = 0; c < NI; ++c) acc += mr[c] * src[c * STRIDE];
    out[e] = acc;
  }
}

template <int D, int NV, int NI, int NO, typename T = double>
__device__ __forceinline__ T* apply_ct(T* a, T* b, const T* M, int tid, int nth) {
  apply_pass_ct<D, NV, NI, NO, 0, T>(a, b, M, tid, nth);
  __syncthreads();
  if (D == 1) return b;
  apply_pass_ct<D, NV, NI, NO, 1, T>(b, a, M, tid, nth);
  __syncthreads();
  if (D == 2) return a;
  apply_pass_ct<D, NV, NI, NO, 2, T>(a, b, M, tid, nth);
  __syncthreads();
  return b;
}

// Block-wide reductions of per-thread values (blockDim a multiple of 32).
__device__ __forceinline__ double block_reduce_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = nanmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double r = red[0];
  for (int i = 1; i < nw; ++i) r = nanmax(r, red[i]);
  __syncthreads();
  return r;
}

__device__ __forceinline__ double block_reduce_min(double v, double* red) {
  return -block_reduce_max(-v, red);
}

// Trace element e of a cell, laid out [k][side][v][ts + NF * m] (face axis k,
// side s, variable v, tangential node ts, time node m): returns v and sets the
// space-time node offset `base` of the line of n nodes across axis k, its
// stride `stk` and the side s.
template <int D, int n>
__device__ __forceinline__ int trace_index(int e, int& base, int& stk, int& s) {
  constexpr int NV = D + 2, ND = ipow(n, D), NF = ipow(n, D - 1), NT = NF * n;
  const int k = e / (2 * NV * NT);
  int r = e - k * (2 * NV * NT);
  s = r / (NV * NT);
  r -= s * (NV * NT);
  const int v = r / NT, tt = r - v * NT;
  const int m = tt / NF;
  int ts = tt - m * NF;
  int st = 1;
  base = m * ND;
  stk = 1;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    if (j == k) {
      stk = st;
    } else {
      base += (ts % n) * st;
      ts /= n;
    }
    st *= n;
  }
  return v;
}

// ---------------------------------------------------------------------------
// K1 predictor: one cell per block.  Writes the candidate's volume part
// u + sum_k c_k Mvol x_k fbar_k into Unext and the space-time face traces.
// ---------------------------------------------------------------------------
template <int D, int N, bool MIXED>
__host__ __device__ constexpr size_t predictor_smem_bytes() {
  using DM = Dims<D, N>;
  size_t d = (size_t)DM::NV * DM::ND + (size_t)DM::NV * DM::NST + (size_t)D * DM::NV * DM::NST +
             (size_t)D * DM::NV * DM::ND + 3 * DM::n * DM::n + 3 * DM::n;
  // the FP32 sweep arrays qf, Ff live inside the FP64 flux array F (unused
  // until the FP32 sweeps are over); u and the trace weights in FP32 stay
  // apart (the FP32 sweep operators are in constant memory)
  size_t f = MIXED ? ((size_t)DM::NV * DM::ND + 2 * DM::n) : 0;
  return d * sizeof(double) + f * sizeof(float);
}

template <int D, int N, bool MIXED>
__global__ void __launch_bounds__(PredShape<D, N, MIXED>::bound, PredShape<D, N, MIXED>::min_blocks)
    k_predictor(Batch bt) {
  using DM = Dims<D, N>;
  constexpr int n = DM::n, NV = DM::NV, ND = DM::ND, NST = DM::NST, NF = DM::NF, NT = DM::NT;
  extern __shared__ double sm[];
  double* u = sm;
  double* q = u + NV * ND;
  double* F = q + NV * NST;
  double* fbar = F + D * NV * NST;
  double* Dm = fbar + D * NV * ND;
  double* Kt = Dm + n * n;
  double* Mv = Kt + n * n;
  double* w = Mv + n * n;
  double* ph0 = w + n;
  double* ph1 = ph0 + n;
  // FP32 sweep arrays inside F: (1 + D) NV NST floats fit in D NV NST doubles
  float* qf = reinterpret_cast<float*>(F);
  float* Ff = qf + NV * NST;
  float* uf = reinterpret_cast<float*>(ph1 + n);
  float* ph0f = uf + NV * ND;
  float* ph1f = ph0f + n;

  const int tid = threadIdx.x, nth = blockDim.x;
  const Ops* o = bt.pps[0]->ops;      // every state of a batch has degree N
  for (int i = tid; i < n * n; i += nth) {
    Dm[i] = o->D[i];
    Kt[i] = o->Kt[i];
    Mv[i] = o->Mvol[i];
  }
  for (int i = tid; i < n; i += nth) {
    w[i] = o->w[i];
    ph0[i] = o->phi0[i];
    ph1[i] = o->phi1[i];
    if (MIXED) {
      ph0f[i] = (float)o->phi0[i];
      ph1f[i] = (float)o->phi1[i];
    }
  }
  for (long long g = blockIdx.x; g < bt.pre[bt.n]; g += gridDim.x) {
    const int sidx = batch_state(bt, g);
    const Params& p = *bt.pps[sidx];
    const long long cell = g - bt.pre[sidx];
    const double dt = *p.b.dt;
    if (!(dt > 0.0)) continue;          // state idle this step (block-uniform)
    double c[3];
#pragma unroll
    for (int k = 0; k < D; ++k) c[k] = p.b.coef[k];
    const double gm1 = p.gamma - 1.0;
    const double* Uc = p.b.U[p.cur] + cell * (NV * ND);
    for (int i = tid; i < NV * ND; i += nth) u[i] = Uc[i];
    __syncthreads();
    int it0 = 0;
    const int n32 = p.iters - p.fp64_sweeps;    // sweeps in FP32
    // with no FP64 sweep the traces split into trace(u) (FP64, once per face
    // node) + trace(q - u) (FP32, per space-time node): the same sum, with
    // FP32 rounding only on the small correction
    const bool split = MIXED && n32 > 0 && p.fp64_sweeps == 0;
    double* tr = p.b.trace + cell * (size_t)(D * 2 * NV * NT);
    if (MIXED && n32 > 0) {
      float cf[3];
#pragma unroll
      for (int k = 0; k < D; ++k) cf[k] = (float)c[k];
      for (int e = tid; e < NV * ND; e += nth) uf[e] = (float)u[e];
      __syncthreads();
      for (int e = tid; e < NV * NST; e += nth) {
        const int v = e / NST, l = e - v * NST;
        qf[e] = uf[v * ND + (l % ND)];
      }
      __syncthreads();
      const bool last64 = p.fp64_sweeps == 0;     // no FP64 sweep: close on the FP64 u
      for (int it = 0; it < n32; ++it) {
        picard_flux<D, n, float>(qf, Ff, (float)gm1, tid, nth);
        __syncthreads();
        picard_deriv_lines<D, N>(Ff, qf, cf, tid, nth);
        __syncthreads();
        if (last64 && it == n32 - 1) picard_time_dq<D, N>(qf, Ff, tid, nth);
        else picard_time_cf<D, N>(qf, uf, tid, nth);
        __syncthreads();
      }
      if (!last64)
        for (int e = tid; e < NV * NST; e += nth) q[e] = (double)qf[e];
      it0 = n32;
    } else {
      for (int e = tid; e < NV * NST; e += nth) {
        const int v = e / NST, l = e - v * NST;
        q[e] = u[v * ND + (l % ND)];
      }
    }
    __syncthreads();
    for (int it = it0; it < p.iters; ++it) {
      picard_flux<D, n, double>(q, F, gm1, tid, nth);
      __syncthreads();
      picard_deriv<D, n, double>(F, q, Dm, c, tid, nth);
      __syncthreads();
      picard_time<D, n, double>(q, u, Kt, tid, nth);
      __syncthreads();
    }
    if (split) {
      // final stage on u (FP64) + dq (FP32): fbar_k = F_k(u) + sum_m w_m
      // (F_k(u + dq_m) - F_k(u)); the face traces stay split, trace(u) in FP64
      // and trace(dq) in FP32 (split trace layout, see k_faceflux)
      const float* dq = Ff;
      float* dF = qf + 2 * NV * NST;      // [D][NV][NST] weighted flux differences
      for (int i = tid; i < ND; i += nth) {
        double Q[NV], Fl[D][D + 2];
#pragma unroll
        for (int v = 0; v < NV; ++v) Q[v] = u[v * ND + i];
        euler_fluxes<D, double>(Q, gm1, Fl);
#pragma unroll
        for (int k = 0; k < D; ++k)
#pragma unroll
          for (int v = 0; v < NV; ++v) fbar[(k * NV + v) * ND + i] = Fl[k][v];
      }
      for (int e = tid; e < D * 2 * NV * NF; e += nth) {
        int base, stk, s;
        const int v = trace_index<D, n>((e / NF) * NT + e % NF, base, stk, s);   // time node 0
        const double* ph = s ? ph1 : ph0;
        double acc = 0.0;
#pragma unroll
        for (int a = 0; a < n; ++a) acc += ph[a] * u[v * ND + base + a * stk];
        tr[(e / (NV * NF)) * (NV * NT) + e % (NV * NF)] = acc;
      }
      for (int l = tid; l < NST; l += nth) {
        const int i = l % ND, m = l / ND;
        float U[NV], dQ[NV], G[D][D + 2];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          U[v] = uf[v * ND + i];
          dQ[v] = dq[v * NST + l];
        }
        euler_flux_delta<D>(U, dQ, (float)gm1, G);
        const float wm = (float)w[m];
#pragma unroll
        for (int k = 0; k < D; ++k)
#pragma unroll
          for (int v = 0; v < NV; ++v) dF[(k * NV + v) * NST + l] = wm * G[k][v];
      }
      __syncthreads();
      for (int e = tid; e < D * 2 * NV * NT; e += nth) {
        int base, stk, s;
        const int v = trace_index<D, n>(e, base, stk, s);
        const float* ph = s ? ph1f : ph0f;
        const float* d = dq + v * NST + base;
        float acc = 0.0f;
#pragma unroll
        for (int a = 0; a < n; ++a) acc += ph[a] * d[a * stk];
        const int blk = e / (NV * NT);
        reinterpret_cast<float*>(tr + blk * (NV * NT) + NV * NF)[e - blk * (NV * NT)] = acc;
      }
      for (int e = tid; e < D * NV * ND; e += nth) {
        const int kv = e / ND, i = e - kv * ND;
        float acc = 0.0f;
#pragma unroll
        for (int m = 0; m < n; ++m) acc += dF[kv * NST + i + m * ND];
        fbar[e] += (double)acc;
      }
    } else {
      // corrector volume term from the time-averaged nodal fluxes
      picard_flux<D, n, double>(q, F, gm1, tid, nth);
      __syncthreads();
      for (int e = tid; e < D * NV * ND; e += nth) {
        const int kv = e / ND, i = e - kv * ND;
        double acc = 0.0;
#pragma unroll
        for (int m = 0; m < n; ++m) acc += w[m] * F[kv * NST + i + m * ND];
        fbar[e] = acc;
      }
    }
    __syncthreads();
    double* Uo = p.b.U[1 - p.cur] + cell * (NV * ND);
    for (int e = tid; e < NV * ND; e += nth) {
      const int v = e / ND, i = e - v * ND;
      double acc = u[e];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const int st = (k == 0) ? 1 : (k == 1 ? n : n * n);
        const int ak = (i / st) % n;
        const double* f = fbar + (k * NV + v) * ND + (i - ak * st);
        double t = 0.0;
#pragma unroll
        for (int j = 0; j < n; ++j) t += Mv[ak * n + j] * f[j * st];
        acc += c[k] * t;
      }
      Uo[e] = acc;
    }
    // space-time traces on the 2D faces: trace[cell][k][side][v][ts + NF * m]
    if (!split)
      for (int e = tid; e < D * 2 * NV * NT; e += nth) {
        int base, stk, s;
        const int v = trace_index<D, n>(e, base, stk, s);
        const double* ph = s ? ph1 : ph0;
        const double* qq = q + v * NST + base;
        double acc = 0.0;
#pragma unroll
        for (int a = 0; a < n; ++a) acc += ph[a] * qq[a * stk];
        tr[e] = acc;
      }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// K2 face flux: the time-averaged numerical flux at every tangential node of
// every face normal to axis k.
// ---------------------------------------------------------------------------
// Whether a state's predictor leaves its face traces split: per (cell, axis,
// side) block of NV x NT doubles, trace(u) [NV][NF] in FP64 followed by
// trace(dq) [NV][NT] in FP32 (mixed precision with no FP64 Picard sweep).
__device__ __forceinline__ bool split_traces(const Params& p) {
  return p.prec == ADG_PREC_MIXED_FP32 && p.fp64_sweeps == 0 && p.iters > 0;
}

// Space-time trace value at tangential node ts, time node m of one block.
template <int D, int n>
__device__ __forceinline__ void load_trace(const double* blk, int ts, int m, bool split, double* Q) {
  constexpr int NV = D + 2, NF = ipow(n, D - 1), NT = NF * n;
  if (split) {
    const float* d = reinterpret_cast<const float*>(blk + NV * NF);
#pragma unroll
    for (int v = 0; v < NV; ++v) Q[v] = blk[v * NF + ts] + (double)d[v * NT + ts + NF * m];
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) Q[v] = blk[v * NT + ts + NF * m];
  }
}

// Euler flux along axis k (FP64); RCP: 1 / rho from rcp_newton (the
// mixed-precision path's split face flux).
template <int D, bool RCP = false>
__device__ __forceinline__ void euler_flux_k(const double* Q, double gm1, int k, double* F) {
  const double r = RCP ? rcp_newton(Q[0]) : 1.0 / Q[0];
  double kin = 0.0;
#pragma unroll
  for (int j = 0; j < D; ++j) kin += Q[1 + j] * Q[1 + j];
  const double p = gm1 * (Q[D + 1] - 0.5 * kin * r);
  const double vk = Q[1 + k] * r;
  F[0] = Q[1 + k];
#pragma unroll
  for (int j = 0; j < D; ++j) F[1 + j] = Q[1 + j] * vk;
  F[1 + k] += p;
  F[D + 1] = vk * (Q[D + 1] + p);
}

// F_k(U + dQ) - F_k(U) in FP32, every term carrying a factor of dQ (the
// along-axis-k part of euler_flux_delta).
template <int D>
__device__ __forceinline__ void euler_flux_delta_k(const float* U, const float* dQ, float gm1, int k,
                                                   float* G) {
  const float r = 1.0f / U[0];
  const float r1 = 1.0f / (U[0] + dQ[0]);
  float v[D], dv[D];
  float mv = 0.0f, dmv = 0.0f;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    v[j] = U[1 + j] * r;
    mv += U[1 + j] * v[j];
    dv[j] = (dQ[1 + j] - v[j] * dQ[0]) * r1;
  }
#pragma unroll
  for (int j = 0; j < D; ++j) dmv += dQ[1 + j] * (v[j] + dv[j]) + U[1 + j] * dv[j];
  const float Ep = U[D + 1] + gm1 * (U[D + 1] - 0.5f * mv);
  const float dp = gm1 * (dQ[D + 1] - 0.5f * dmv);
  const float vk1 = v[k] + dv[k];
  G[0] = dQ[1 + k];
#pragma unroll
  for (int j = 0; j < D; ++j) G[1 + j] = dQ[1 + j] * vk1 + U[1 + j] * dv[k];
  G[1 + k] += dp;
  G[D + 1] = (dQ[D + 1] + dp) * vk1 + Ep * dv[k];
}

// |v_k| + c of U + dQ in FP32, with rho p = (gamma - 1)(E rho - |m|^2 / 2)
// taken as the FP64 value rpU of U plus its change, which carries a factor of
// dQ; NaN for an inadmissible state.
template <int D>
__device__ __forceinline__ float speed_split(const float* U, const float* dQ, float rpU, float gamma,
                                             float gm1, int k) {
  float drp = U[D + 1] * dQ[0] + (U[0] + dQ[0]) * dQ[D + 1];
#pragma unroll
  for (int j = 0; j < D; ++j) drp -= (U[1 + j] + 0.5f * dQ[1 + j]) * dQ[1 + j];
  const float r = 1.0f / (U[0] + dQ[0]);
  return fabsf(U[1 + k] + dQ[1 + k]) * r + sqrtf(gamma * (rpU + gm1 * drp)) * r;
}

// Time-averaged Rusanov flux of an interior face from split traces:
//   G = (F_k(uL) + F_k(uR)) / 2 + sum_m w_m (dF_L,m + dF_R,m) / 2
//       - (uR - uL) sum_m w_m s_m / 2 - sum_m w_m s_m (dqR_m - dqL_m) / 2,
// F_k(u) in FP64 once per face node, the per-time-node parts in FP32.
template <int D, int n>
__device__ __forceinline__ void face_split_rusanov(const double* bL, const double* bR, int ts, int k,
                                                   double gamma, const float* wf, float gf,
                                                   float gm1f, double* G) {
  constexpr int NV = D + 2, NF = ipow(n, D - 1), NT = NF * n;
  const float* dL = reinterpret_cast<const float*>(bL + NV * NF);
  const float* dR = reinterpret_cast<const float*>(bR + NV * NF);
  const double gm1 = gamma - 1.0;
  double uL[NV], uR[NV], FL[NV], FR[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    uL[v] = bL[v * NF + ts];
    uR[v] = bR[v * NF + ts];
  }
  euler_flux_k<D, true>(uL, gm1, k, FL);
  euler_flux_k<D, true>(uR, gm1, k, FR);
  double kinL = 0.0, kinR = 0.0;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    kinL += uL[1 + j] * uL[1 + j];
    kinR += uR[1 + j] * uR[1 + j];
  }
  // the FP32 copies of the FP64 terms, narrowed on the integer pipe (toward
  // zero: they are the base states of the FP32 per-time-node corrections)
  const float rpL = narrow_f64_rz(gm1 * (uL[D + 1] * uL[0] - 0.5 * kinL));
  const float rpR = narrow_f64_rz(gm1 * (uR[D + 1] * uR[0] - 0.5 * kinR));
  float ULf[NV], URf[NV], sumD[NV], sumJ[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    ULf[v] = narrow_f64_rz(uL[v]);
    URf[v] = narrow_f64_rz(uR[v]);
    sumD[v] = 0.0f;
    sumJ[v] = 0.0f;
  }
  float S = 0.0f;
#pragma unroll 1
  for (int m = 0; m < n; ++m) {
    float qL[NV], qR[NV], GL[NV], GR[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      qL[v] = dL[v * NT + ts + NF * m];
      qR[v] = dR[v * NT + ts + NF * m];
    }
    euler_flux_delta_k<D>(ULf, qL, gm1f, k, GL);
    euler_flux_delta_k<D>(URf, qR, gm1f, k, GR);
    const float sL = speed_split<D>(ULf, qL, rpL, gf, gm1f, k);
    const float sR = speed_split<D>(URf, qR, rpR, gf, gm1f, k);
    const float s = (sL > sR || sL != sL) ? sL : sR;     // NaN propagates
    const float wm = wf[m];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      sumD[v] += wm * (GL[v] + GR[v]);
      sumJ[v] += wm * s * (qR[v] - qL[v]);
    }
    S += wm * s;
  }
  const double Sd = widen_f32(S);
#pragma unroll
  for (int v = 0; v < NV; ++v)
    G[v] = 0.5 * (FL[v] + FR[v]) + 0.5 * widen_f32(sumD[v]) -
           0.5 * ((uR[v] - uL[v]) * Sd + widen_f32(sumJ[v]));
}

// One thread per (face, tangential node): the Rusanov (or Osher-type) flux at
// each time node, weighted by the time rule.  At a domain boundary the missing
// side is the ghost state of the face's kind (boundary_ghost).
template <int D, int N>
__global__ void __launch_bounds__(256, 2) k_faceflux(Batch bt, int k) {
  using DM = Dims<D, N>;
  constexpr int n = DM::n, NV = DM::NV, NF = DM::NF, NT = DM::NT;
  for (long long eg = blockIdx.x * (long long)blockDim.x + threadIdx.x; eg < bt.pre[bt.n];
       eg += (long long)gridDim.x * blockDim.x) {
    const int sidx = batch_state(bt, eg);
    const Params& p = *bt.pps[sidx];
    if (!(*p.b.dt > 0.0)) continue;
    const long long e = eg - bt.pre[sidx];
    const Geo& g = p.geo;
    const double* w = p.ops->w;
    double* G = p.b.G[k];
    const long long face = e / NF;
    const int ts = (int)(e - face * NF);
    int ijk[3] = {0, 0, 0};
    long long r = face;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const int ext = (j == k) ? g.n[j] + 1 : g.n[j];
      ijk[j] = (int)(r % ext);
      r /= ext;
    }
    const int f = ijk[k];
    int L[3], R[3];
#pragma unroll
    for (int j = 0; j < D; ++j) L[j] = R[j] = ijk[j];
    bool hasL = true, hasR = true;
    if (f == 0) {
      if (g.periodic[k]) L[k] = g.n[k] - 1; else hasL = false;
    } else {
      L[k] = f - 1;
    }
    if (f == g.n[k]) {
      if (g.periodic[k]) R[k] = 0; else hasR = false;
    }
    const size_t csz = (size_t)D * 2 * NV * NT;
    const double* trL = hasL ? p.b.trace + cell_index<D>(L, g) * csz + ((size_t)k * 2 + 1) * NV * NT
                             : nullptr;
    const double* trR = hasR ? p.b.trace + cell_index<D>(R, g) * csz + ((size_t)k * 2 + 0) * NV * NT
                             : nullptr;
    if (!hasL) trL = trR;
    if (!hasR) trR = trL;
    const bool split = split_traces(p);
    double acc[NV];
    if (split && hasL && hasR && p.flux == ADG_FLUX_RUSANOV) {
      face_split_rusanov<D, n>(trL, trR, ts, k, p.gamma, p.ops->wf, p.b.coef_f[7], p.b.coef_f[6], acc);
#pragma unroll
      for (int v = 0; v < NV; ++v) G[(face * NV + v) * NF + ts] = acc[v];
      continue;
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.0;
    for (int m = 0; m < n; ++m) {
      double QL[NV], QR[NV], Gm[NV];
      load_trace<D, n>(trL, ts, m, split, QL);
      load_trace<D, n>(trR, ts, m, split, QR);
      if (!hasL || !hasR) {
        const int face = 2 * k + (hasL ? 1 : 0);
        double pos = 0.0, t = 0.0;
        if (g.bc[face] == ADG_BC_FRONT) {
          // the node's coordinate along the front's axis, and its time
          const int j = g.front_axis[face];
          int a = 0, tt = ts;
#pragma unroll
          for (int jj = 0; jj < D; ++jj)
            if (jj != k) {
              if (jj == j) a = tt % n;
              tt /= n;
            }
          pos = g.x0[j] + (ijk[j] + p.ops->xi[a]) * g.dx[j];
          t = *p.b.tstart + p.ops->xi[m] * *p.b.dt;
        }
        if (!hasL) boundary_ghost<D>(g, face, QR, QL, pos, t);
        else boundary_ghost<D>(g, face, QL, QR, pos, t);
      }
      face_flux<D>(p.flux, QL, QR, k, p.gamma, Gm, p.prec == ADG_PREC_MIXED_FP32);
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] += w[m] * Gm[v];
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) G[(face * NV + v) * NF + ts] = acc[v];
  }
}

// Tangential node index of spatial node i for the faces normal to axis k.
template <int D, int n>
__device__ __forceinline__ int tangential(int i, int k) {
  int ts = 0, mul = 1;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const int a = i % n;
    i /= n;
    if (j != k) {
      ts += a * mul;
      mul *= n;
    }
  }
  return ts;
}

// Order-preserving map of a double onto a signed 64-bit key (x < y <=> key(x)
// < key(y) for non-NaN x, y; +NaN above +inf), so that min / max reductions
// run on the integer pipe instead of the FP64 pipe.
__device__ __forceinline__ long long ord_key(double x) {
  const long long b = __double_as_longlong(x);
  return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double ord_val(long long k) {
  return __longlong_as_double(k >= 0 ? k : (k ^ 0x7fffffffffffffffLL));
}
// max(a, b) of two doubles that are not negative (+0 included) and not NaN:
// their bit patterns order as signed integers
__device__ __forceinline__ double max_nonneg(double a, double b) {
  return __double_as_longlong(a) >= __double_as_longlong(b) ? a : b;
}
// Bulk prefetch of `bytes` (a multiple of 16, 16-byte aligned) into L2 by the
// TMA unit (cp.async.bulk.prefetch): no shared memory, nothing to wait for.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Bulk prefetch into L2 of the 16-byte-aligned part of [src, src + bytes), in
// pieces of at most 4 KB (the bytes outside it, at most 15 at each end, are
// left to the loads).
__device__ __forceinline__ void prefetch_range_l2(const void* src, size_t bytes) {
  const uintptr_t a = (reinterpret_cast<uintptr_t>(src) + 15) & ~(uintptr_t)15;
  const uintptr_t e = (reinterpret_cast<uintptr_t>(src) + bytes) & ~(uintptr_t)15;
  for (uintptr_t x = a; x < e; x += 4096) {
    const uintptr_t len = (e - x < 4096) ? (e - x) : 4096;
    bulk_prefetch_l2(reinterpret_cast<const void*>(x), (unsigned)len);
  }
}

// Key of a wave speed for a max-reduction: a NaN of either sign (an
// inadmissible state) is the largest key, so the cell's speed is NaN and the
// CFL step reports the state (ord_key alone would order a NaN with its sign
// bit set below every speed).
__device__ __forceinline__ long long speed_key(double s) {
  return isnan_f64(s) ? LLONG_MAX : ord_key(s);
}

// Detector bounds over the Voronoi neighbourhood (3^d block) from per-cell
// min/max, then the relaxed DMP interval [m - delta, M + delta] (Eq. relax
// with a relative floor).  Threads v < nvar write lohi[2v], lohi[2v+1].
template <int D>
__device__ __forceinline__ void dmp_interval_lane(const Params& p, const double* __restrict__ cmm,
                                                  const int* ijk, double* lohi, int v);

template <int D>
__device__ __forceinline__ void dmp_interval(const Params& p, const double* __restrict__ cmm,
                                             const int* ijk, double* lohi) {
  if ((int)threadIdx.x < D + 2) dmp_interval_lane<D>(p, cmm, ijk, lohi, threadIdx.x);
}

// The interval of variable v (one thread per variable).
template <int D>
__device__ __forceinline__ void dmp_interval_lane(const Params& p, const double* __restrict__ cmm,
                                                  const int* ijk, double* lohi, int v) {
  const int NV = D + 2;
  const Geo& g = p.geo;
  // min / max on order-preserving integer keys (the integer pipe), NaNs
  // skipped as fmin / fmax skip them
  long long kmn = LLONG_MAX, kmx = LLONG_MIN;
  const int nb3 = ipow(3, D);
  for (int o = 0; o < nb3; ++o) {
    int c[3] = {0, 0, 0}, oo = o;
    bool in = true, flip = false;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      int cj = ijk[j] + (oo % 3) - 1;
      oo /= 3;
      if (cj < 0 || cj >= g.n[j]) {
        const int kind = g.bc[2 * j + (cj < 0 ? 0 : 1)];
        if (kind == ADG_BC_PERIODIC) {
          cj = (cj + g.n[j]) % g.n[j];
        } else if (kind == ADG_BC_REFLECTIVE) {
          // mirror image of the boundary cell: its wall-normal momentum
          // bounds negate and swap
          cj = cj < 0 ? 0 : g.n[j] - 1;
          if (v == 1 + j) flip = !flip;
        } else {
          in = false;
        }
      }
      c[j] = cj;
    }
    if (!in) continue;
    const long long nb = cell_index<D>(c, g);
    const double lo = cmm[(nb * NV + v) * 2 + 0], hi = cmm[(nb * NV + v) * 2 + 1];
    // the mirror image's bounds: negated (sign bit) and swapped
    const double l2 = flip ? __longlong_as_double(__double_as_longlong(hi) ^ LLONG_MIN) : lo;
    const double h2 = flip ? __longlong_as_double(__double_as_longlong(lo) ^ LLONG_MIN) : hi;
    if (!isnan_f64(l2)) kmn = min(kmn, ord_key(l2));
    if (!isnan_f64(h2)) kmx = max(kmx, ord_key(h2));
  }
  const double mn = kmn == LLONG_MAX ? INFINITY : ord_val(kmn);
  const double mx = kmx == LLONG_MIN ? -INFINITY : ord_val(kmx);
  // fmax of non-negative doubles as integer compares of their bit patterns
  // (the same result; the FP64 pipe runs fmax)
  const double scale = max_nonneg(1.0, max_nonneg(fabs(mx), fabs(mn)));
  const double delta = max_nonneg(p.eps * (mx - mn), p.floor * scale);
  lohi[2 * v] = mn - delta;
  lohi[2 * v + 1] = mx + delta;
}

// Max-reduces K integer keys per thread over the block (blockDim a multiple of
// 32, at most 256 threads); the results land in red[nw * K + j].
template <int K>
__device__ __forceinline__ const long long* block_max_keys(long long* r, long long* red) {
#pragma unroll
  for (int j = 0; j < K; ++j)
    for (int o = 16; o > 0; o >>= 1) r[j] = max(r[j], __shfl_xor_sync(0xffffffffu, r[j], o));
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int j = 0; j < K; ++j) red[w * K + j] = r[j];
  __syncthreads();
  if (threadIdx.x < K) {
    long long x = red[threadIdx.x];
    for (int i = 1; i < nw; ++i) x = max(x, red[i * K + threadIdx.x]);
    red[nw * K + threadIdx.x] = x;
  }
  __syncthreads();
  return red + nw * K;
}

// Checks the subcell data vs[v][s] of one cell.
//   PAD: rho > 0 and rho E - |m|^2 / 2 > 0 on every subcell (for rho > 0 the
//        second test is p > 0 without a division; NaN in any component fails);
//   DMP (lohi != null): every subcell inside [lo_v, hi_v], tested exactly on
//        the per-variable extremes (min >= lo and max <= hi).
// Writes the per-variable min / max to mm[2v], mm[2v+1] and, when lam != null,
// the largest wave speed max_k |v_k| + c (FP32 speeds with f32speed).  Returns
// (block-uniform) whether any check failed.  `red` needs (blockDim/32 + 1) * (2 nvar + 1) doubles.
template <int D>
__device__ __forceinline__ bool check_subcells(const double* __restrict__ vs, int nsub,
                                               const double* lohi, double gamma, double* mm,
                                               double* lam, double* red, bool f32speed = false,
                                               float g2f = 0.0f) {
  constexpr int NV = D + 2, K = 2 * NV + 1;
  bool bad = false;
  long long r[K];
#pragma unroll
  for (int j = 0; j < K; ++j) r[j] = LLONG_MIN;
  for (int s = threadIdx.x; s < nsub; s += blockDim.x) {
    double Q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      Q[v] = vs[v * nsub + s];
      const long long k = ord_key(Q[v]);
      r[2 * v] = max(r[2 * v], ~k);          // ~k reverses the order: max of ~k = ~min k
      r[2 * v + 1] = max(r[2 * v + 1], k);
    }
    double kin = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) kin += Q[1 + k] * Q[1 + k];
    const double pe = Q[D + 1] * Q[0] - 0.5 * kin;
    // the two PAD comparisons as exact integer tests
    bad = bad || !(positive_f64(Q[0]) && positive_f64(pe));
    if (lam)
      r[2 * NV] = max(r[2 * NV], speed_key(f32speed ? wave_speed_f<D>(Q, pe, g2f) : wave_speed<D>(Q, gamma)));
  }
  bad = __syncthreads_or(bad);
  const long long* res = block_max_keys<K>(r, reinterpret_cast<long long*>(red));
  double mn[NV], mx[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    mn[v] = ord_val(~res[2 * v]);
    mx[v] = ord_val(res[2 * v + 1]);
  }
  if (lohi) {
    // the DMP test on the extremes, by one warp (the others would repeat it)
    int dmp = 0;
    if (threadIdx.x < 32) {
#pragma unroll
      for (int v = 0; v < NV; ++v)
        dmp |= !((mn[v] >= lohi[2 * v]) && (mx[v] <= lohi[2 * v + 1]));
    }
    bad = __syncthreads_or(bad || dmp);
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      mm[2 * v] = mn[v];
      mm[2 * v + 1] = mx[v];
    }
    if (lam) *lam = ord_val(res[2 * NV]);
  }
  return bad;
}

// ---------------------------------------------------------------------------
// K3 + K4 corrector and detector: one cell per block.
// ---------------------------------------------------------------------------
template <int D, int N>
__host__ __device__ constexpr size_t correct_smem_bytes() {
  using DM = Dims<D, N>;
  const int big = DM::NSD > DM::ND * 4 ? DM::NSD : DM::ND * 4;
  // + the face terms' weights (2 d n doubles) and the FP32 copy of P1 (Ns n
  // floats) for the projection of the step's change
  return (size_t)(2 * DM::NV * (DM::NSD > big ? DM::NSD : big) + DM::Ns * DM::n + 4 * DM::NV + 128 +
                  2 * D * DM::n + (DM::Ns * DM::n + 1) / 2) *
         sizeof(double);
}

// (at most 64 registers, eight blocks per SM: 5-12% faster than the 72 the
// compiler takes unbounded)
template <int D, int N>
__global__ void __launch_bounds__(128, 8) k_correct_detect(Batch bt) {
  using DM = Dims<D, N>;
  constexpr int n = DM::n, NV = DM::NV, ND = DM::ND, NF = DM::NF, Ns = DM::Ns, NSD = DM::NSD;
  constexpr int BUF = (DM::NSD > DM::ND * 4 ? DM::NSD : DM::ND * 4);
  extern __shared__ double sm[];
  double* A = sm;                     // NV * BUF
  double* B = A + NV * BUF;           // NV * BUF
  double* P1 = B + NV * BUF;          // Ns * n
  double* lohi = P1 + Ns * n;         // 2 NV
  double* mm = lohi + 2 * NV;         // 2 NV
  double* red = mm + 2 * NV;          // 128
  double* cw = red + 128;             // 2 D n: [k][side][a] dt/dx_k phi_side(a) / w_a
  float* P1f = reinterpret_cast<float*>(cw + 2 * D * n);   // Ns * n
  const int tid = threadIdx.x, nth = blockDim.x;
  const Ops* o = bt.pps[0]->ops;
  for (int i = tid; i < Ns * n; i += nth) {
    P1[i] = o->P1[i];
    P1f[i] = (float)o->P1[i];
  }
  __syncthreads();
  for (long long g = blockIdx.x; g < bt.pre[bt.n]; g += gridDim.x) {
    const int sidx = batch_state(bt, g);
    const Params& p = *bt.pps[sidx];
    const long long cell = g - bt.pre[sidx];
    if (tid == 0) {
      // the next cell's DOF blocks and kept averages, into L2 while this one runs
      const long long gn = g + gridDim.x;
      if (gn < bt.pre[bt.n]) {
        const int sn = batch_state(bt, gn);
        const Params* pn = bt.pps[sn];
        const long long cn = gn - bt.pre[sn];
        prefetch_range_l2(pn->b.U[1 - pn->cur] + cn * (NV * ND), NV * ND * sizeof(double));
        if (pn->b.vstar) {
          prefetch_range_l2(pn->b.U[pn->cur] + cn * (NV * ND), NV * ND * sizeof(double));
          prefetch_range_l2(pn->b.vstar + cn * (size_t)(NV * NSD), NV * NSD * sizeof(double));
        }
      }
    }
    const double dt = *p.b.dt;
    if (!(dt > 0.0)) continue;
    double c[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < D; ++k) c[k] = p.b.coef[k];
    const int nxt = 1 - p.cur;
    int ijk[3];
    cell_coords<D>(cell, p.geo, ijk);
    double* Uo = p.b.U[nxt] + cell * (NV * ND);
    // mixed precision: P(u*) = P(u^n) (kept) + P(u* - u^n) in FP32 where P(u^n)
    // is known, except every 16th step (bounds the drift of the kept values)
    double* vkeep = p.b.vstar ? p.b.vstar + cell * (size_t)(NV * NSD) : nullptr;
    const bool delta = vkeep && p.b.vok[cell] && (p.stamp & 15) != 0;
    const double* Un = p.b.U[p.cur] + cell * (NV * ND);
    float* dA = reinterpret_cast<float*>(B);          // FP32 change, then its projection
    float* dB = dA + NV * BUF;
    // the face terms' weights of this cell's step, one product each (the
    // previous cell's readers passed several barriers since)
    for (int q = tid; q < 2 * D * n; q += nth) {
      const int k = q / (2 * n), r = q - k * 2 * n;
      const double ck = k == 0 ? c[0] : (k == 1 ? c[1] : c[2]);
      cw[q] = ck * (r < n ? o->phi0w[r] : o->phi1w[r - n]);
    }
    __syncthreads();
    for (int e = tid; e < NV * ND; e += nth) {
      const int v = e / ND, i = e - v * ND;
      double acc = Uo[e];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const int st = (k == 0) ? 1 : (k == 1 ? n : n * n);
        const int ak = (i / st) % n;
        const int ts = tangential<D, n>(i, k);
        const long long flo = face_index<D>(p.geo, ijk, k, ijk[k]);
        const long long fhi = face_index<D>(p.geo, ijk, k, ijk[k] + 1);
        const double Glo = p.b.G[k][(flo * NV + v) * NF + ts];
        const double Ghi = p.b.G[k][(fhi * NV + v) * NF + ts];
        // u* -= dt/dx_k (phi1(a)/w_a Ghi - phi0(a)/w_a Glo), as two FMAs
        acc = fma(-cw[(2 * k + 1) * n + ak], Ghi, acc);
        acc = fma(cw[2 * k * n + ak], Glo, acc);
      }
      A[e] = acc;
      Uo[e] = acc;
      if (delta) dA[e] = narrow_f64_rz(acc - Un[e]);    // (integer pipe; toward zero)
    }
    __syncthreads();
    double* vs;
    if (delta) {
      const float* dv = apply_ct<D, NV, n, Ns, float>(dA, dB, P1f, tid, nth);
      for (int e = tid; e < NV * NSD; e += nth) {
        const double x = vkeep[e] + widen_f32(dv[e]);
        A[e] = x;
        vkeep[e] = x;
      }
      vs = A;
    } else {
      vs = apply_ct<D, NV, n, Ns>(A, B, P1, tid, nth);
      if (vkeep)
        for (int e = tid; e < NV * NSD; e += nth) vkeep[e] = vs[e];
    }
    dmp_interval<D>(p, p.b.cmm[p.cur], ijk, lohi);
    __syncthreads();
    double lam = 0.0;
    const bool bad = check_subcells<D>(vs, NSD, lohi, p.gamma, mm, p.lam_mode ? &lam : nullptr, red,
                                       p.prec == ADG_PREC_MIXED_FP32, p.gam2f);
    if (tid == 0) {
      int slot = -1;
      if (bad || p.force) {
        slot = atomicAdd(&p.b.counters[CNT_TROUBLED0 + nxt], 1);
        if (slot < p.cap) {
          p.b.list[nxt][slot] = (int)cell;
        } else {
          // no subcell slot left: the cell keeps its candidate, the step is
          // reported as failed (ADG_ERR_CAPACITY) by the next status query
          atomicOr(&p.b.counters[CNT_STATUS], 1);
          slot = -1;
        }
      }
      p.b.beta[nxt][cell] = (uint8_t)(slot >= 0);
      p.b.slot[nxt][cell] = slot;
      if (p.lam_mode) p.b.lam[cell] = lam;
      if (vkeep) p.b.vok[cell] = 1;       // reset by any later change of the cell's DOFs
    }
    if (tid < 2 * NV) p.b.cmm[nxt][cell * 2 * NV + tid] = mm[tid];
    __syncthreads();
  }
}

}  // namespace adg

namespace adg {

// ---------------------------------------------------------------------------
// K3 + K4 with one warp per cell: the same per-item arithmetic as
// k_correct_detect (face terms, projection, kept averages, PAD, DMP on the
// extremes, integer-key reductions), synchronised by __syncwarp and reduced
// with warp shuffles instead of block barriers; W cells per block.
// ---------------------------------------------------------------------------
constexpr int CD_WARPS = 4;

template <int D, int NV, int NI, int NO, typename T>
__device__ __forceinline__ T* apply_ct_warp(T* a, T* b, const T* M, int lane) {
  apply_pass_ct<D, NV, NI, NO, 0, T>(a, b, M, lane, 32);
  __syncwarp();
  if (D == 1) return b;
  apply_pass_ct<D, NV, NI, NO, 1, T>(b, a, M, lane, 32);
  __syncwarp();
  if (D == 2) return a;
  apply_pass_ct<D, NV, NI, NO, 2, T>(a, b, M, lane, 32);
  __syncwarp();
  return b;
}

// Warp version of check_subcells: per-variable extremes, PAD, the DMP test on
// the extremes against lohi (if given) and the largest wave speed; every lane
// returns the results (mm[2v], mm[2v+1], *lam) and whether a check failed.
template <int D>
__device__ __forceinline__ bool check_subcells_warp(const double* __restrict__ vs, int nsub,
                                                    const double* lohi, double gamma, double* mm,
                                                    double* lam, bool f32speed, int lane,
                                                    float g2f) {
  constexpr int NV = D + 2, K = 2 * NV + 1;
  bool bad = false;
  long long r[K];
#pragma unroll
  for (int j = 0; j < K; ++j) r[j] = LLONG_MIN;
  for (int s = lane; s < nsub; s += 32) {
    double Q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      Q[v] = vs[v * nsub + s];
      const long long k = ord_key(Q[v]);
      r[2 * v] = max(r[2 * v], ~k);
      r[2 * v + 1] = max(r[2 * v + 1], k);
    }
    double kin = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) kin += Q[1 + k] * Q[1 + k];
    const double pe = Q[D + 1] * Q[0] - 0.5 * kin;
    bad = bad || !(positive_f64(Q[0]) && positive_f64(pe));
    if (lam)
      r[2 * NV] = max(r[2 * NV], speed_key(f32speed ? wave_speed_f<D>(Q, pe, g2f) : wave_speed<D>(Q, gamma)));
  }
#pragma unroll
  for (int j = 0; j < K; ++j)
    for (int o = 16; o > 0; o >>= 1) r[j] = max(r[j], __shfl_xor_sync(0xffffffffu, r[j], o));
  bad = __any_sync(0xffffffffu, bad);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    mm[2 * v] = ord_val(~r[2 * v]);
    mm[2 * v + 1] = ord_val(r[2 * v + 1]);
  }
  if (lohi) {
#pragma unroll
    for (int v = 0; v < NV; ++v)
      bad = bad || !((mm[2 * v] >= lohi[2 * v]) && (mm[2 * v + 1] <= lohi[2 * v + 1]));
  }
  if (lam) *lam = ord_val(r[2 * NV]);
  return bad;
}

template <int D, int N>
struct CdLayout {
  using DM = Dims<D, N>;
  // sizes per variable of the projection's stages: u (n^D), after the x pass
  // (Ns n^(D-1)), after the y pass (Ns^2 n^(D-2)), after the z pass (Ns^3)
  static constexpr int S0 = DM::ND, S1 = DM::Ns * ipow(DM::n, D - 1);
  static constexpr int S2 = (D >= 2) ? DM::Ns * DM::Ns * ipow(DM::n, D - 2) : 0;
  static constexpr int S3 = (D == 3) ? DM::NSD : 0;
  static constexpr int SA = S0 > S2 ? S0 : S2, SB = S1 > S3 ? S1 : S3;
  // per warp: A [NV][SA] doubles (u*, then P(u*)), B (the FP64 projection's
  // other stage, [NV][SB] doubles, or the FP32 projection of the change:
  // [NV][SA] + [NV][SB] floats), face weights [2 D][n] doubles, lohi [2 NV]
  static constexpr int A_DBL = DM::NV * SA;
  static constexpr int B_DBL = (DM::NV * SB > (DM::NV * (SA + SB) + 1) / 2) ? DM::NV * SB
                                                                            : (DM::NV * (SA + SB) + 1) / 2;
  static constexpr int DB_FLT = DM::NV * SA;          // offset of the second FP32 stage
  static constexpr int CW_DBL = 2 * D * DM::n;
  static constexpr int WARP_DBL = A_DBL + B_DBL + CW_DBL + 2 * DM::NV;
  // per block: P1 [Ns n] doubles and its FP32 copy
  static constexpr int OPS_DBL = DM::Ns * DM::n + (DM::Ns * DM::n + 1) / 2;
};

template <int D, int N>
__host__ __device__ constexpr size_t correct_warp_smem_bytes() {
  return (size_t)(CdLayout<D, N>::OPS_DBL + CD_WARPS * CdLayout<D, N>::WARP_DBL) * sizeof(double);
}

template <int D, int N>
__global__ void __launch_bounds__(32 * CD_WARPS) k_correct_detect_w(Batch bt) {
  using DM = Dims<D, N>;
  using LY = CdLayout<D, N>;
  constexpr int n = DM::n, NV = DM::NV, ND = DM::ND, NF = DM::NF, Ns = DM::Ns, NSD = DM::NSD;
  extern __shared__ double sm[];
  double* P1 = sm;
  float* P1f = reinterpret_cast<float*>(P1 + Ns * n);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double* A = sm + LY::OPS_DBL + w * LY::WARP_DBL;
  double* B = A + LY::A_DBL;
  double* cw = B + LY::B_DBL;          // [k][side][a]: dt/dx_k phi_side(a) / w_a
  double* lohi = cw + LY::CW_DBL;
  const Ops* o = bt.pps[0]->ops;
  for (int i = threadIdx.x; i < Ns * n; i += 32 * CD_WARPS) {
    P1[i] = o->P1[i];
    P1f[i] = (float)o->P1[i];
  }
  __syncthreads();
  const long long total = bt.pre[bt.n];
  for (long long g = (long long)blockIdx.x * CD_WARPS + w; g < total;
       g += (long long)gridDim.x * CD_WARPS) {
    const int sidx = batch_state(bt, g);
    const Params& p = *bt.pps[sidx];
    const long long cell = g - bt.pre[sidx];
    if (lane == 0) {
      // the next cell's DOF blocks and kept averages, into L2 while this one runs
      const long long gn = g + (long long)gridDim.x * CD_WARPS;
      if (gn < total) {
        const int sn = batch_state(bt, gn);
        const Params* pn = bt.pps[sn];
        const long long cn = gn - bt.pre[sn];
        constexpr unsigned UB = NV * ND * sizeof(double), VB = NV * NSD * sizeof(double);
        static_assert(UB % 16 == 0 && VB % 16 == 0, "bulk prefetch sizes are multiples of 16 bytes");
        bulk_prefetch_l2(pn->b.U[1 - pn->cur] + cn * (NV * ND), UB);
        if (pn->b.vstar) {
          bulk_prefetch_l2(pn->b.U[pn->cur] + cn * (NV * ND), UB);
          bulk_prefetch_l2(pn->b.vstar + cn * (size_t)(NV * NSD), VB);
        }
      }
    }
    const double dt = *p.b.dt;
    if (!(dt > 0.0)) continue;          // (warp-uniform)
    double c[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < D; ++k) c[k] = p.b.coef[k];
    const int nxt = 1 - p.cur;
    int ijk[3];
    cell_coords<D>(cell, p.geo, ijk);
    double* Uo = p.b.U[nxt] + cell * (NV * ND);
    double* vkeep = p.b.vstar ? p.b.vstar + cell * (size_t)(NV * NSD) : nullptr;
    const bool delta = vkeep && p.b.vok[cell] && (p.stamp & 15) != 0;
    const double* Un = p.b.U[p.cur] + cell * (NV * ND);
    float* dA = reinterpret_cast<float*>(B);
    float* dB = dA + LY::DB_FLT;
    // the face terms' weights of this cell's step, one product each
    for (int q = lane; q < 2 * D * n; q += 32) {
      const int k = q / (2 * n), r = q - k * 2 * n;
      const double ck = k == 0 ? c[0] : (k == 1 ? c[1] : c[2]);   // (registers, not a local array)
      cw[q] = ck * (r < n ? o->phi0w[r] : o->phi1w[r - n]);
    }
    __syncwarp();
    for (int e = lane; e < NV * ND; e += 32) {
      const int v = e / ND, i = e - v * ND;
      double acc = Uo[e];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const int st = (k == 0) ? 1 : (k == 1 ? n : n * n);
        const int ak = (i / st) % n;
        const int ts = tangential<D, n>(i, k);
        const long long flo = face_index<D>(p.geo, ijk, k, ijk[k]);
        const long long fhi = face_index<D>(p.geo, ijk, k, ijk[k] + 1);
        const double Glo = p.b.G[k][(flo * NV + v) * NF + ts];
        const double Ghi = p.b.G[k][(fhi * NV + v) * NF + ts];
        // u* -= dt/dx_k (phi1(a)/w_a Ghi - phi0(a)/w_a Glo), as two FMAs
        acc = fma(-cw[(2 * k + 1) * n + ak], Ghi, acc);
        acc = fma(cw[2 * k * n + ak], Glo, acc);
      }
      A[e] = acc;
      Uo[e] = acc;
      if (delta) dA[e] = narrow_f64_rz(acc - Un[e]);
    }
    __syncwarp();
    double* vs;
    if (delta) {
      const float* dv = apply_ct_warp<D, NV, n, Ns, float>(dA, dB, P1f, lane);
      for (int e = lane; e < NV * NSD; e += 32) {
        const double x = vkeep[e] + widen_f32(dv[e]);
        A[e] = x;
        vkeep[e] = x;
      }
      vs = A;
    } else {
      vs = apply_ct_warp<D, NV, n, Ns, double>(A, B, P1, lane);
      if (vkeep)
        for (int e = lane; e < NV * NSD; e += 32) vkeep[e] = vs[e];
    }
    if (lane < NV) dmp_interval_lane<D>(p, p.b.cmm[p.cur], ijk, lohi, lane);
    __syncwarp();
    double lam = 0.0, mm[2 * NV];
    const bool bad = check_subcells_warp<D>(vs, NSD, lohi, p.gamma, mm, p.lam_mode ? &lam : nullptr,
                                            p.prec == ADG_PREC_MIXED_FP32, lane, p.gam2f);
    if (lane == 0) {
      int slot = -1;
      if (bad || p.force) {
        slot = atomicAdd(&p.b.counters[CNT_TROUBLED0 + nxt], 1);
        if (slot < p.cap) {
          p.b.list[nxt][slot] = (int)cell;
        } else {
          atomicOr(&p.b.counters[CNT_STATUS], 1);
          slot = -1;
        }
      }
      p.b.beta[nxt][cell] = (uint8_t)(slot >= 0);
      p.b.slot[nxt][cell] = slot;
      if (p.lam_mode) p.b.lam[cell] = lam;
      if (vkeep) p.b.vok[cell] = 1;
    }
#pragma unroll
    for (int j = 0; j < 2 * NV; ++j)
      if (lane == j) p.b.cmm[nxt][cell * 2 * NV + j] = mm[j];
    __syncwarp();
  }
}

}  // namespace adg
