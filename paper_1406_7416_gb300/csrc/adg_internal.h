// Internal declarations of libadg: operator tables, grid geometry, device
// buffers, Euler physics and the kernel launch interface.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/adg.h"

namespace adg {

constexpr int MAXN = 10;              // nodes per axis, n = N + 1 <= 10
constexpr int MAXNS = 19;             // subcells per axis, Ns = 2N + 1 <= 19
constexpr double WENO_EPS = 1e-14;    // WENO3 weights: lambda_k / (sigma_k + eps)^8
constexpr double WENO_LAMBDA_C = 1e5; // central stencil; side stencils use 1

// 1D operators of the degree-N nodal Gauss-Legendre basis on [0, 1] and of the
// degree-2 subcell basis, generated on the host (ops_host.cpp) and copied to
// the device once per state.
struct Ops {
  int N, n, Ns;
  double xi[MAXN], w[MAXN];
  double D[MAXN * MAXN];      // D[a*n+b]  = phi_b'(xi_a)
  double Kt[MAXN * MAXN];     // Ktau[m*n+j] = (K1^{-1} diag(w))[m][j]
  double phi0[MAXN], phi1[MAXN];
  double phi0w[MAXN], phi1w[MAXN];   // phi(0)/w, phi(1)/w
  double Mvol[MAXN * MAXN];   // Mvol[a*n+j] = w_j D[j][a] / w_a
  double P1[MAXNS * MAXN];    // P1[s*n+a]   subcell averages of phi_a
  double R1[MAXN * MAXNS];    // R1[a*Ns+s]  (P1^T P1)^{-1} P1^T
  double Mt[MAXN * MAXNS];    // Mt[b*Ns+e]  = P1[e][b] / (Ns w_b)
  // composite rule for the initial data: Ns subintervals x (N+2) points
  double cq_x[MAXNS * (MAXN + 1)], cq_w[MAXNS * (MAXN + 1)];
  double cq_phi[MAXNS * (MAXN + 1) * MAXN];   // phi_a(cq_x[p]) at [p*n+a]
  // degree-2 subcell basis (3 GL nodes)
  double w3[3], xi3[3], D3[9], Kt3[9], phi03[3], phi13[3];
  // WENO3: coefficient matrices C[k][p*3+r] (stencil k, monomial p, cell r),
  // nodal evaluation E[j*3+p] = xi3_j^p
  double C[3][9];
  double E[9];
  // float copies for the reduced-precision Picard sweeps
  float Df[MAXN * MAXN], Ktf[MAXN * MAXN];
  float wf[MAXN];             // time weights in FP32 (the split face fluxes)
  // FP32 WENO3 (mixed precision): per stencil k the rows of C for c1, c2
  // (Cf[k][0..2], Cf[k][3..5]) and the nodal values straight from the stencil
  // averages, Wf[k][node * 3 + r] = sum_p E[node][p] C[k][p][r]
  float Cf[3][6];
  float Wf[3][9];
};

// Builds the operator table of degree N (host, long double arithmetic).
void build_ops(int N, Ops* ops);

struct Geo {
  int dim;
  int n[3];
  int periodic[3];
  int bc[6];             // boundary kind (ADG_BC_*) of face 2k (low) / 2k+1 (high) of axis k
  double x0[3];
  double dx[3];
  double bstate[6][5];   // conserved state of every ADG_BC_INFLOW face
  // ADG_BC_FRONT faces: split at x_axis = a + b t; part 0 before, part 1 after
  int front_axis[6];
  int front_kind[6][2];
  double front_a[6], front_b[6];
  double front_state[6][2][5];
  long long cells;
};

// Per-state device buffers.  Index [cur] holds time level n, [1-cur] level n+1.
struct Bufs {
  double* U[2];          // [cells][nv][n^d]
  uint8_t* beta[2];      // [cells]
  double* cmm[2];        // [cells][nv][2]  per-cell min / max of the subcell data
  int* slot[2];          // [cells] slot of a troubled cell, -1 otherwise
  int* list[2];          // [cap]   cell of each slot
  double* store[2];      // [cap][nv][Ns^d] subcell data v of troubled cells
  double* trace;         // [cells][d][2][nv][n^(d-1) * n]
  double* G[3];          // per axis [faces][nv][n^(d-1)], time-averaged DG face flux
  double* lam;           // [cells] max wave speed over the cell's subcell data
  int* counters;         // see CNT_*
  int* fixlist;          // [cells]
  int* fixstamp;         // [cells]
  double* edge;          // [cap][d][2][nv][Ns^(d-1)] sub-face fluxes on the cell faces
  int* hist;             // [HIST_LEN] troubled count of step s at s % HIST_LEN (s from 0)
  int* fblist;           // [cap] slots whose WENO3 result failed PAD this step
  int* fbflag;           // [cap] step stamp of the slots in fblist
  int* refixlist;        // [cap] WENO3 cells sharing a face with a fallback cell
  double* dt;            // [1] time step of the current step (0: state idle this step)
  double* lamred;        // [1] reduced lambda
  long long* lamkey;     // [1] bits of the largest per-cell wave speed (CFL steps; 0 between steps)
  double* clock;         // [3] simulated time t, end time t_end (0: none), steps taken
  double* tstart;        // [1] simulated time at the start of the current step
  double* coef;          // [6] dt / dx_k and dt Ns / dx_k of the current step (set once per step)
  float* coef_f;         // [8] FP32 copies for the FP32 subcell kernels: coef[0..5], gamma - 1,
                         // gamma (conversions from FP64 run on the narrow FP64 pipe)
  // mixed precision, ADG_OPT_PROJECT_DELTA: the subcell averages P(u) of each
  // cell's current DOFs, kept from the detector of the step that made them
  double* vstar;         // [cells][nv][Ns^d] (null when off)
  uint8_t* vok;          // [cells] 1 where vstar is P of the cell's current DOFs
  // limiter scratch, sized for one chunk of `chunk` troubled cells
  double* patch;         // [chunk][nv][L^d]
  double* sweep[3];      // [chunk][nv][...] after the x, y, z reconstructions
  double* qsub;          // [chunk][(Ns+2)^d][nv][3^(d+1)]
  double* fsub[3];       // [chunk][nv][faces along axis k]
  double* tmp_sub;       // load-time scratch [cells][nv][Ns^d]
};

constexpr int HIST_LEN = 4096;        // steps of troubled-count history kept per state

enum {
  CNT_TROUBLED0 = 0,     // troubled count of buffer 0
  CNT_TROUBLED1 = 1,     // troubled count of buffer 1
  CNT_FIX = 2,           // neighbour-fix list length
  CNT_STATUS = 3,        // bit 0: slot capacity exceeded, bit 1: bad dt
  CNT_INADM = 4,         // subcells left inadmissible after the limiter
  CNT_FB = 5,            // first-order fallback cells of the current step
  CNT_REFIX = 6,         // WENO3 cells rebalanced against a fallback neighbour
  CNT_FB_TOTAL = 7,      // fallback cells since the last load
  CNT_PASSES = 8,        // limiter passes run by device-sized pass loops (cumulative)
  CNT_COUNT = 9
};

struct Params {
  Geo geo;
  int N, dim, nv, prec, iters, force, cap, chunk;
  double gamma, eps, floor;
  const Ops* ops;        // device copy
  Bufs b;
  int cur;               // buffer index of time level n
  int stamp;             // step counter (fix-list stamps)
  int lam_mode;          // 1: kernels keep the per-cell wave speeds current
  int fp64_sweeps;       // mixed precision: number of final FP64 Picard sweeps
  int cascade;           // 1: first-order layer after WENO3 (Sec. 6, Fig. algo2)
  int flux;              // numerical flux of DG faces and WENO3 sub-faces: 0 Rusanov, 1 Osher
  double cfl;            // the state's CFL number for batched CFL steps (0: none)
  float gam2f;           // gamma (gamma - 1) in FP32: the mixed-precision wave speed's factor
};

// A batch of states of one (dimension, degree, precision) stepped by the same
// launches.  Each state's Params lives in device memory (pps[s]); `pre` is the
// item prefix of the launch (pre[s] = first item of state s, pre[n] = total).
struct Batch {
  Params* const* pps;
  int n;
  const long long* pre;
};

// state owning item g: pre[s] <= g < pre[s+1]
__device__ __forceinline__ int batch_state(const Batch& b, long long g) {
  int lo = 0, hi = b.n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (b.pre[mid] <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Device descriptors of one batched step (all arrays in device memory).
struct StepLaunch {
  Params* const* pps;          // [n] per-state device Params
  int n;
  const long long* pre_cells;  // [n+1]
  const long long* pre_faces[3];  // [n+1] faces x tangential nodes, per axis
  long long* pre_lim;          // [n+3] troubled cells of one limiter pass (device-computed);
                               // [n+1] the pass, [n+2] passes needed (device-sized loops)
  long long* pre_fix;          // [n+1] neighbour-fix entries (device-computed)
  long long* pre_fb;           // [n+1] first-order fallback cells (device-computed)
  long long* pre_refix;        // [n+1] rebalanced WENO3 neighbours (device-computed)
  int cascade;                 // any state of the launch runs the first-order layer
  int sub32;                   // mixed precision: FP32 sweeps (of 3) of the subcell predictor
  int sub_f32;                  // mixed precision: WENO3 reconstruction and sub-face fluxes in FP32
  int sub_reg;                 // the FP32 subcell predictor with a subcell in one warp's registers
  int flux;                    // numerical flux of the launch's states (ADG_FLUX_*)
  int pred;                    // predictor launch shape (PRED_*)
  long long total_cells;
  long long total_faces[3];
  long long sum_chunk;         // sum over states of the limiter chunk size
  int max_passes;              // max over states of ceil(capacity / chunk)
  int prec;
  cudaEvent_t* ev;             // phase events or null
  const double* dts;           // [n] fixed steps, or null for CFL steps
  double cfl;                  // CFL number when dts is null
  double dt_max;               // cap of CFL steps (<= 0: none)
  // device-sized limiter passes (stream capture only): the pass body is the
  // child graph of a conditional WHILE node on `cond`, captured on `body`
  int loop;
  cudaGraphConditionalHandle cond;
  cudaStream_t body;
};

// Launch shapes of the predictor (selected per state by the autotuner or the
// ADG_OPT_PREDICTOR option; every shape computes the same outputs):
//   PRED_BLOCK      one block per cell (k_predictor), its default threads;
//   PRED_BLOCK_ALT  one block per cell at the other block width (256 threads
//                   where the default is 128 or 160, 128 where it is 256; the
//                   FP32 kernels whose default is their launch bound: 64);
//   PRED_WARP1/2/4  mixed precision with the split final stage: one warp per
//                   cell for the FP32 sweeps, 1, 2 or 4 cells per block sharing
//                   the FP64 terms (k_predictor_split);
//   PRED_WARP4_TC   the same with the sweeps' contractions on the tensor pipe
//                   (3 x TF32 mma.sync, FP32-accurate).
enum PredShapeId { PRED_BLOCK = 0, PRED_BLOCK_ALT = 1, PRED_WARP2 = 2, PRED_WARP4 = 3,
                   PRED_WARP4_TC = 4, PRED_WARP1 = 5, PRED_COUNT = 6 };

// Kernel launch interface: one dispatcher per translation unit (2D low N,
// 2D high N, 3D), selected by dimension and degree.
enum LaunchOp {
  OP_STEP_BEGIN = 10,  // per-state dt (fixed or CFL), counters, stamps
  OP_STEP_END = 11,    // per-state level swap
  OP_STEP_DG = 0,      // predictor, face fluxes, corrector + detector
  OP_STEP_LIMITER,     // subcell limiter over the troubled list + flux correction
  OP_LOAD_DETECT,      // initial detection (exact may be null)
  OP_LOAD_FULL,        // full-state load
  OP_READ_FULL,        // subcell rows of flagged cells
  OP_PROJECT,          // initial data projection
  OP_SUB_MINMAX,       // per-cell min/max of subcell rows
  OP_LAMBDA,           // per-cell wave speeds of the current level
  OP_PREDICTOR,        // the predictor alone (autotuning), shape step->pred
  OP_PACK,             // halo exchange: a box of cells into a buffer
  OP_UNPACK            // halo exchange: a buffer into a box of cells, list rebuilt
};

struct LaunchArgs {
  int op;
  const Params* p;
  cudaStream_t stream;
  const double* exact;     // OP_LOAD_DETECT: exact averages (device) or null
  const double* cmm_ex;    // OP_LOAD_DETECT: their per-cell min/max
  const uint8_t* beta;     // OP_LOAD_FULL
  const double* sub;       // OP_LOAD_FULL input, OP_SUB_MINMAX input
  double* out;             // OP_READ_FULL rows, OP_PROJECT exact averages, OP_SUB_MINMAX result
  const adg_problem* prob; // OP_PROJECT
  const double* fac;       // OP_PROJECT per-cell density factor (device) or null
  cudaEvent_t* ev;         // unused (phase events travel in StepLaunch)
  const StepLaunch* step;  // OP_STEP_*: the batched step
  const int* box;          // OP_PACK / OP_UNPACK: lo[3], hi[3] (host)
  void* buf;               // OP_PACK / OP_UNPACK: the packed cells (device)
};

// Bytes of a packed box of `count` cells (halo exchange).
size_t packed_bytes(int dim, int N, long long count);

// Phase boundaries recorded when profiling is on: ev[PHASE_x] before phase x,
// ev[PHASE_END] after the last one.
enum { PHASE_PREDICTOR = 0, PHASE_FACEFLUX, PHASE_CORRECT, PHASE_LIMITER, PHASE_FIX, PHASE_END,
       PHASE_COUNT };

cudaError_t dispatch_2d_lo(int N, const LaunchArgs& a);   // N = 1..5
cudaError_t dispatch_2d_hi(int N, const LaunchArgs& a);   // N = 6..9
cudaError_t dispatch_3d(int N, const LaunchArgs& a);      // N = 1..3
// FP32 Picard operators of degree N into the constant memory of the unit
// that launches that (dimension, degree)
cudaError_t upload_constants_2d_lo(int N, const Ops& o);
cudaError_t upload_constants_2d_hi(int N, const Ops& o);
cudaError_t upload_constants_3d(int N, const Ops& o);
cudaError_t launch_dt(const Params& p, double cfl, double dt_max, cudaStream_t s);
cudaError_t launch_set_scalar(double* dst, double v, cudaStream_t s);
// dimension-independent batch kernels (k3d.cu)
cudaError_t launch_step_begin(const StepLaunch& sl, cudaStream_t s);
cudaError_t launch_step_end(const StepLaunch& sl, cudaStream_t s);
cudaError_t launch_lim_prefix(const StepLaunch& sl, int pass, cudaStream_t s);
cudaError_t launch_fix_prefix(const StepLaunch& sl, cudaStream_t s);
cudaError_t launch_count_prefix(const StepLaunch& sl, long long* pre, int counter, cudaStream_t s);
// Device-sized limiter passes in a captured graph: `begin` sizes the loop from
// the troubled counts and opens it, then `add_loop_node` appends the WHILE node
// to the capture on `s` and returns its (empty) body graph; the body ends with
// `next`, which advances the pass and closes the loop after the last one.
cudaError_t launch_lim_loop_begin(const StepLaunch& sl, cudaStream_t s);
cudaError_t launch_lim_loop_next(const StepLaunch& sl, cudaStream_t s);
cudaError_t add_loop_node(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraph_t* body);

// Scratch doubles per troubled cell of the limiter chunk buffers.
size_t limiter_scratch_doubles(int dim, int N, size_t* patch, size_t* sw0, size_t* sw1,
                               size_t* sw2, size_t* qsub, size_t* fsub);

// ---------------------------------------------------------------------------
// Euler physics (Sec. 5): conserved (rho, rho v, rho E), ideal gas.
// ---------------------------------------------------------------------------
template <int D, typename T>
__device__ __forceinline__ void euler_fluxes(const T* Q, T gm1, T (*F)[D + 2]) {
  const T r = T(1) / Q[0];
  T v[D];
  T kin = T(0);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    v[k] = Q[1 + k] * r;
    kin += Q[1 + k] * v[k];
  }
  const T p = gm1 * (Q[D + 1] - T(0.5) * kin);
  const T Ep = Q[D + 1] + p;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    F[k][0] = Q[1 + k];
#pragma unroll
    for (int j = 0; j < D; ++j) F[k][1 + j] = Q[1 + j] * v[k];
    F[k][1 + k] += p;
    F[k][D + 1] = v[k] * Ep;
  }
}

// Conversions and tests on the integer pipe.  GB300 runs every FP64
// instruction -- conversions between FP32 and FP64 and FP64 comparisons
// included -- on its narrow FP64 pipe (about the rate of an FP64 FMA, measured),
// so the kernels whose FP64 work bounds them use these bit-level forms.

#if defined(__CUDACC__)
// x > 0, exactly the FP64 comparison (false for NaN, +0 and -0).
__device__ __forceinline__ bool positive_f64(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b <= 0x7ff0000000000000LL;
}

__device__ __forceinline__ bool isnan_f64(double x) {
  return (__double_as_longlong(x) & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL;
}

// FP32 -> FP64 widening: exact for normal numbers, infinities and NaNs; FP32
// subnormals (|x| < 2^-126) become zeros of their sign.
__device__ __forceinline__ double widen_f32(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned s = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  if (e == 0) return __hiloint2double((int)s, 0);
  const unsigned e11 = (e == 0xffu) ? 0x7ffu : e + 896u;   // rebias 127 -> 1023
  return __hiloint2double((int)(s | (e11 << 20) | (m >> 3)), (int)(m << 29));
}

// FP64 -> FP32 narrowing toward zero: the top 23 mantissa bits; magnitudes
// below the FP32 normal range give zeros of their sign, above it the largest
// finite float; infinities stay, NaNs stay NaN.
__device__ __forceinline__ float narrow_f64_rz(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned s = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  if (e == 0x7ff) return __uint_as_float(s | ((((hi & 0xfffffu) | lo) != 0u) ? 0x7fc00000u : 0x7f800000u));
  const int e8 = e - 896;
  if (e8 <= 0) return __uint_as_float(s);
  if (e8 >= 255) return __uint_as_float(s | 0x7f7fffffu);
  return __uint_as_float(s | ((unsigned)e8 << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}

// 1 / x in FP64 by the Newton-Raphson iteration for the reciprocal,
// r <- r + r (1 - x r) (the error squares at every step), from an FP32 seed
// formed off the FP64 pipe (integer-pipe narrowing, FP32 reciprocal,
// integer-pipe widening): two FP64 steps take its ~2^-22 relative error below
// FP64 rounding.  For x whose FP32 narrowing is a normal number the result is
// within 1 ulp of 1.0 / x (adg_pipe_rates checks this on the device); zeros,
// infinities, NaNs and magnitudes outside the FP32 normal range are outside
// that promise.  Used by the mixed-precision path's split face flux only (in
// the predictor's FP64 terms, which are not FP64-pipe bound, it was slower
// than the division: 3.58 against 3.49 ms at 512^2, N = 5).
__device__ __forceinline__ double rcp_newton(double x) {
  double r = widen_f32(__frcp_rn(narrow_f64_rz(x)));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

#endif

__device__ __forceinline__ double nanmax(double a, double b) {
  // max that propagates NaN from either argument
  return (a > b || a != a) ? a : b;
}

template <int D>
__device__ __forceinline__ double euler_pressure(const double* Q, double gm1) {
  double kin = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) kin += Q[1 + k] * Q[1 + k];
  return gm1 * (Q[D + 1] - 0.5 * kin / Q[0]);
}

// Rusanov flux through a face with normal +e_k, pointwise (Sec. 2.3).  With
// f32speed (mixed precision) the sound speeds take an FP32 square root: the
// speed only scales the dissipation term s (QR - QL), so its FP32 rounding
// is relative to the jump, and the flux stays single-valued.
template <int D>
__device__ __forceinline__ void rusanov(const double* QL, const double* QR, int k, double gamma,
                                        double* G, bool f32speed = false) {
  const double gm1 = gamma - 1.0;
  double sL, sR, FL[D + 2], FR[D + 2];
  {
    const double r = 1.0 / QL[0];
    double kin = 0.0;
#pragma unroll
    for (int j = 0; j < D; ++j) kin += QL[1 + j] * QL[1 + j];
    const double p = gm1 * (QL[D + 1] - 0.5 * kin * r);
    const double vk = QL[1 + k] * r;
    sL = fabs(vk) + (f32speed ? (double)sqrtf((float)(gamma * p * r)) : sqrt(gamma * p * r));
    FL[0] = QL[1 + k];
#pragma unroll
    for (int j = 0; j < D; ++j) FL[1 + j] = QL[1 + j] * vk;
    FL[1 + k] += p;
    FL[D + 1] = vk * (QL[D + 1] + p);
  }
  {
    const double r = 1.0 / QR[0];
    double kin = 0.0;
#pragma unroll
    for (int j = 0; j < D; ++j) kin += QR[1 + j] * QR[1 + j];
    const double p = gm1 * (QR[D + 1] - 0.5 * kin * r);
    const double vk = QR[1 + k] * r;
    sR = fabs(vk) + (f32speed ? (double)sqrtf((float)(gamma * p * r)) : sqrt(gamma * p * r));
    FR[0] = QR[1 + k];
#pragma unroll
    for (int j = 0; j < D; ++j) FR[1 + j] = QR[1 + j] * vk;
    FR[1 + k] += p;
    FR[D + 1] = vk * (QR[D + 1] + p);
  }
  const double s = nanmax(sL, sR);
#pragma unroll
  for (int v = 0; v < D + 2; ++v) G[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * s * (QR[v] - QL[v]);
}

// Universal Osher-type flux of Dumbser and Toro through a face with normal
// +e_k (Sec. 2.3 names it; it is the flux of the vortex table of Sec. 5.2):
//   G = (F(QL) + F(QR))/2 - (1/2) sum_j w_j |A_k(psi_j)| (QR - QL)
// on the straight path psi(s) = QL + s (QR - QL), three-point Gauss-Legendre
// rule in s.  |A_k| dQ = sum_m |lambda_m| alpha_m r_m, with the right
// eigenvectors r_m of A_k at psi_j and the wave strengths alpha = R^{-1} dQ
// in closed form (normal velocity u = v_k, tangential components v_t):
//   alpha_t = dm_t - v_t drho,   dE' = dE - sum_t alpha_t v_t,
//   alpha_0 = (gamma-1)/c^2 (drho (H - u^2) + u dm_k - dE'),
//   alpha_- = (drho (u + c) - dm_k - c alpha_0) / (2c),
//   alpha_+ = drho - alpha_- - alpha_0,
//   r_- = (1, v - c e_k, H - u c), r_0 = (1, v, |v|^2/2), r_t = (0, e_t, v_t),
//   r_+ = (1, v + c e_k, H + u c); eigenvalues u - c, u (d times), u + c.
template <int D>
__device__ __forceinline__ void osher(const double* QL, const double* QR, int k, double gamma,
                                      double* G) {
  constexpr int NV = D + 2;
  const double gm1 = gamma - 1.0;
  double dQ[NV], acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    dQ[v] = QR[v] - QL[v];
    acc[v] = 0.0;
  }
  const double half_span = 0.38729833462074168852;       // sqrt(3/5) / 2
  const double sj[3] = {0.5 - half_span, 0.5, 0.5 + half_span};
  const double wj[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    double Q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Q[v] = QL[v] + sj[j] * dQ[v];
    const double r = 1.0 / Q[0];
    double vel[D], kin = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      vel[a] = Q[1 + a] * r;
      kin += vel[a] * vel[a];
    }
    const double p = gm1 * (Q[D + 1] - 0.5 * Q[0] * kin);
    const double c2 = gamma * p * r;
    const double c = sqrt(c2);
    const double H = (Q[D + 1] + p) * r;
    const double u = vel[k];
    double dE = dQ[D + 1];
    double at[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      at[a] = (a == k) ? 0.0 : dQ[1 + a] - vel[a] * dQ[0];
      dE -= at[a] * vel[a];
    }
    const double a0 = gm1 / c2 * (dQ[0] * (H - u * u) + u * dQ[1 + k] - dE);
    const double am = (dQ[0] * (u + c) - dQ[1 + k] - c * a0) / (2.0 * c);
    const double ap = dQ[0] - am - a0;
    const double lm = wj[j] * fabs(u - c) * am;
    const double l0 = wj[j] * fabs(u);
    const double lp = wj[j] * fabs(u + c) * ap;
    acc[0] += lm + l0 * a0 + lp;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      double m = (lm + lp + l0 * a0) * vel[a] + l0 * at[a];
      if (a == k) m += (lp - lm) * c;
      acc[1 + a] += m;
    }
    double e = lm * (H - u * c) + lp * (H + u * c) + l0 * a0 * 0.5 * kin;
#pragma unroll
    for (int a = 0; a < D; ++a) e += l0 * at[a] * vel[a];
    acc[D + 1] += e;
  }
  double FL[NV], FR[NV];
  {
    const double r = 1.0 / QL[0];
    double kin = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) kin += QL[1 + a] * QL[1 + a];
    const double p = gm1 * (QL[D + 1] - 0.5 * kin * r);
    const double vk = QL[1 + k] * r;
    FL[0] = QL[1 + k];
#pragma unroll
    for (int a = 0; a < D; ++a) FL[1 + a] = QL[1 + a] * vk;
    FL[1 + k] += p;
    FL[D + 1] = vk * (QL[D + 1] + p);
  }
  {
    const double r = 1.0 / QR[0];
    double kin = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) kin += QR[1 + a] * QR[1 + a];
    const double p = gm1 * (QR[D + 1] - 0.5 * kin * r);
    const double vk = QR[1 + k] * r;
    FR[0] = QR[1 + k];
#pragma unroll
    for (int a = 0; a < D; ++a) FR[1 + a] = QR[1 + a] * vk;
    FR[1 + k] += p;
    FR[D + 1] = vk * (QR[D + 1] + p);
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) G[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * acc[v];
}

// FP32 Rusanov flux (mixed-precision sub-faces), the same formulas as rusanov.
template <int D>
__device__ __forceinline__ void rusanov_f(const float* QL, const float* QR, int k, float gamma,
                                          float* G) {
  const float gm1 = gamma - 1.0f;
  float s[2], F[2][D + 2];
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const float* Q = side ? QR : QL;
    const float r = 1.0f / Q[0];
    float kin = 0.0f;
#pragma unroll
    for (int j = 0; j < D; ++j) kin += Q[1 + j] * Q[1 + j];
    const float p = gm1 * (Q[D + 1] - 0.5f * kin * r);
    const float vk = Q[1 + k] * r;
    s[side] = fabsf(vk) + sqrtf(gamma * p * r);
    F[side][0] = Q[1 + k];
#pragma unroll
    for (int j = 0; j < D; ++j) F[side][1 + j] = Q[1 + j] * vk;
    F[side][1 + k] += p;
    F[side][D + 1] = vk * (Q[D + 1] + p);
  }
  const float sm = (s[0] > s[1] || s[0] != s[0]) ? s[0] : s[1];   // NaN propagates
#pragma unroll
  for (int v = 0; v < D + 2; ++v) G[v] = 0.5f * (F[0][v] + F[1][v]) - 0.5f * sm * (QR[v] - QL[v]);
}

// The numerical flux selected by the state's option (0 Rusanov, 1 Osher-type).
template <int D>
__device__ __forceinline__ void face_flux(int which, const double* QL, const double* QR, int k,
                                          double gamma, double* G, bool f32speed = false) {
  if (which == 1) osher<D>(QL, QR, k, gamma, G);
  else rusanov<D>(QL, QR, k, gamma, G, f32speed);
}

// max_k |v_k| + c of one state (wave speed for Eq. cfl)
template <int D>
__device__ __forceinline__ double wave_speed(const double* Q, double gamma) {
  const double r = 1.0 / Q[0];
  double kin = 0.0, vm = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    kin += Q[1 + k] * Q[1 + k];
    vm = nanmax(vm, fabs(Q[1 + k] * r));
  }
  const double p = (gamma - 1.0) * (Q[D + 1] - 0.5 * kin * r);
  return vm + sqrt(gamma * p * r);
}

// The same speed for mixed precision (it only sets the CFL step): pe =
// E rho - |m|^2 / 2 comes from the caller in FP64 (free of the cancellation
// FP32 would suffer at high Mach numbers; the caller tests it for
// positivity), then c = sqrt(gamma (gamma - 1) pe) / rho with g2f =
// gamma (gamma - 1) and the velocities in FP32, from inputs narrowed toward
// zero on the integer pipe.  Inadmissible states give NaN as in wave_speed.
#if defined(__CUDACC__)
template <int D>
__device__ __forceinline__ double wave_speed_f(const double* Q, double pe, float g2f) {
  const float r = 1.0f / narrow_f64_rz(Q[0]);
  float vm = 0.0f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const float a = fabsf(narrow_f64_rz(Q[1 + k])) * r;
    vm = (a > vm || a != a) ? a : vm;
  }
  return widen_f32(vm + sqrtf(g2f * narrow_f64_rz(pe)) * r);
}
#endif

// ---------------------------------------------------------------------------
// Grid helpers
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void cell_coords(long long c, const Geo& g, int* ijk) {
  ijk[0] = (int)(c % g.n[0]);
  long long r = c / g.n[0];
  if (D == 3) {
    ijk[1] = (int)(r % g.n[1]);
    ijk[2] = (int)(r / g.n[1]);
  } else {
    ijk[1] = (int)r;
  }
}

template <int D>
__device__ __forceinline__ long long cell_index(const int* ijk, const Geo& g) {
  long long c = ijk[0] + (long long)g.n[0] * ijk[1];
  if (D == 3) c += (long long)g.n[0] * g.n[1] * ijk[2];
  return c;
}

// Neighbour across the low (side = -1) or high (side = +1) face of axis k.
// Returns false outside a transmissive boundary.
template <int D>
__device__ __forceinline__ bool face_neighbour(const Geo& g, const int* ijk, int k, int side,
                                               int* out) {
#pragma unroll
  for (int j = 0; j < D; ++j) out[j] = ijk[j];
  int c = ijk[k] + side;
  if (c < 0 || c >= g.n[k]) {
    if (!g.periodic[k]) return false;
    c = (c + g.n[k]) % g.n[k];
  }
  out[k] = c;
  return true;
}

// Ghost state of one boundary kind for the interior state Q at a face normal
// to axis k: transmissive a copy (zero-gradient), reflective the mirror image
// (wall-normal momentum negated), inflow the fixed state q.
template <int D>
__device__ __forceinline__ void ghost_of_kind(int kind, int k, const double* q, const double* Q,
                                              double* G) {
  if (kind == ADG_BC_INFLOW) {
#pragma unroll
    for (int v = 0; v < D + 2; ++v) G[v] = q[v];
    return;
  }
#pragma unroll
  for (int v = 0; v < D + 2; ++v) G[v] = Q[v];
  if (kind == ADG_BC_REFLECTIVE) G[1 + k] = -G[1 + k];
}

// Part (0 before, 1 after) of front face `face` at coordinate pos along the
// front's axis and time t.
__device__ __forceinline__ int front_part(const Geo& g, int face, double pos, double t) {
  return pos < g.front_a[face] + g.front_b[face] * t ? 0 : 1;
}

// Ghost state beyond boundary face `face` (2k low, 2k+1 high of axis k) for
// the interior state Q at the same point; a front face picks its part by the
// point's coordinate `pos` along the front's axis and the time t.  Not used
// for periodic faces.
template <int D>
__device__ __forceinline__ void boundary_ghost(const Geo& g, int face, const double* Q, double* G,
                                               double pos = 0.0, double t = 0.0) {
  int kind = g.bc[face];
  const double* q = g.bstate[face];
  if (kind == ADG_BC_FRONT) {
    const int part = front_part(g, face, pos, t);
    kind = g.front_kind[face][part];
    q = g.front_state[face][part];
  }
  ghost_of_kind<D>(kind, face >> 1, q, Q, G);
}

// Face index along axis k: faces (n_k + 1) along k, cells along the others.
template <int D>
__device__ __forceinline__ long long face_index(const Geo& g, const int* ijk, int k, int f) {
  long long idx = 0, stride = 1;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const int e = (j == k) ? g.n[j] + 1 : g.n[j];
    const int c = (j == k) ? f : ijk[j];
    idx += stride * c;
    stride *= e;
  }
  return idx;
}

template <int D>
__host__ __device__ __forceinline__ long long face_count(const Geo& g, int k) {
  long long c = 1;
  for (int j = 0; j < D; ++j) c *= (j == k) ? g.n[j] + 1 : g.n[j];
  return c;
}

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

}  // namespace adg
