// Subcell limiter kernels (Sec. 4.3-4.4): gather of the subcell patch from
// Eq. (ader.icbc), dimension-by-dimension WENO3 reconstruction, degree-2
// space-time predictor per subcell, sub-face Rusanov fluxes, finite volume
// update A (Eq. aderweno), reconstruction R (Eq. subcell.r) and the flux
// correction of unlimited face neighbours.  All work runs over the compacted
// troubled-cell list, in chunks of `chunk` cells that share the scratch.
#pragma once

#include "kernels_dg.cuh"

namespace adg {

__host__ __device__ __forceinline__ int ipow3(int k) { return k == 0 ? 1 : (k == 1 ? 3 : (k == 2 ? 9 : 27)); }

// Troubled cells handled by limiter pass `pass` of one state (0 past the end,
// and 0 for a state idle this step).  Pass c covers list entries
// [c * chunk, (c + 1) * chunk).
__device__ __forceinline__ int pass_len(const Params& p, int pass) {
  if (!(*p.b.dt > 0.0)) return 0;
  int nT = p.b.counters[CNT_TROUBLED0 + (1 - p.cur)];
  if (nT > p.cap) nT = p.cap;
  const int len = nT - pass * p.chunk;
  return len < 0 ? 0 : (len > p.chunk ? p.chunk : len);
}

// The pass a limiter kernel works on: its argument, or for the pass loop
// sized on the device (argument < 0) the pass stored after the prefix.
__device__ __forceinline__ int lim_pass(const Batch& bt, int pass) {
  return pass >= 0 ? pass : (int)bt.pre[bt.n + 1];
}

// Item t (a troubled cell of the current pass, counted over the batch) ->
// state index and the cell's position j within its state's pass.
struct LimItem {
  int s;
  int j;
};
__device__ __forceinline__ LimItem lim_item(const Batch& bt, long long t) {
  LimItem it;
  it.s = batch_state(bt, t);
  it.j = (int)(t - bt.pre[it.s]);
  return it;
}

// v^n at one subcell of cell `o` (Eq. ader.icbc): the stored subgrid data of a
// troubled cell, else the projection P(u^n) evaluated at that subcell.
template <int D, int N>
__device__ __forceinline__ void subcell_value(const Params& p, long long o, const int* s,
                                              const double* __restrict__ P1, double* out) {
  using DM = Dims<D, N>;
  constexpr int n = DM::n, NV = DM::NV, ND = DM::ND, Ns = DM::Ns, NSD = DM::NSD;
  if (p.b.beta[p.cur][o]) {
    const int slot = p.b.slot[p.cur][o];
    const int sidx = s[0] + Ns * (s[1] + (D == 3 ? Ns * s[2] : 0));
    const double* st = p.b.store[p.cur] + (size_t)slot * NV * NSD;
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v] = st[v * NSD + sidx];
    return;
  }
  const double* U = p.b.U[p.cur] + o * (NV * ND);
  const double* px = P1 + s[0] * n;
  const double* py = P1 + s[1] * n;
  const double* pz = P1 + (D == 3 ? s[2] : 0) * n;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const double* Uv = U + v * ND;
    double acc = 0.0;
    for (int c = 0; c < (D == 3 ? n : 1); ++c) {
      double accb = 0.0;
      for (int b = 0; b < n; ++b) {
        double acca = 0.0;
#pragma unroll
        for (int a = 0; a < n; ++a) acca += px[a] * Uv[a + n * (b + n * c)];
        accb += py[b] * acca;
      }
      acc += (D == 3 ? pz[c] : 1.0) * accb;
    }
    out[v] = acc;
  }
}

// v^n at local subcell loc[k] (may lie outside the cell, up to three
// layers) around cell ijk, with the ghost rules of the boundary kinds: a
// global subcell index outside the domain wraps (periodic), is clamped
// (transmissive: constant extrapolation), is mirrored with the wall-normal
// momentum negated (reflective: -1 - g below, 2 n - 1 - g above), or takes
// the face's fixed state (inflow).  The per-axis transforms apply in axis
// order.
template <int D, int N>
__device__ __forceinline__ void patch_value(const Params& p, const int* ijk, const int* loc,
                                            const double* __restrict__ P1, double* val) {
  using DM = Dims<D, N>;
  constexpr int NV = DM::NV, Ns = DM::Ns;
  const Geo& g = p.geo;
  int own[3] = {0, 0, 0}, sub[3] = {0, 0, 0}, mode[3] = {0, 0, 0};
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const int ng = g.n[k] * Ns;
    int gi = ijk[k] * Ns + loc[k];
    if (gi < 0 || gi >= ng) {
      const int face = 2 * k + (gi < 0 ? 0 : 1);
      int kind = g.bc[face];
      int part = -1;
      if (kind == ADG_BC_FRONT) {
        // the ghost subcell's centre along the front's axis (unmapped index)
        const int j = g.front_axis[face];
        const double h = g.dx[j] / Ns;
        const double pos = g.x0[j] + ((ijk[j] * Ns + loc[j]) + 0.5) * h;
        part = front_part(g, face, pos, *p.b.tstart);
        kind = g.front_kind[face][part];
      }
      if (kind == ADG_BC_PERIODIC) {
        gi = (gi % ng + ng) % ng;
      } else {
        if (kind == ADG_BC_REFLECTIVE) {
          gi = gi < 0 ? -1 - gi : 2 * ng - 1 - gi;
          mode[k] = 1;
        } else if (kind == ADG_BC_INFLOW) {
          // which fixed state: 2 + 2 face an inflow face's, 14 + 2 face + part a front part's
          mode[k] = (part < 0) ? 2 + 2 * face : 14 + 2 * face + part;
        }
        gi = gi < 0 ? 0 : (gi >= ng ? ng - 1 : gi);
      }
    }
    own[k] = gi / Ns;
    sub[k] = gi - own[k] * Ns;
  }
  subcell_value<D, N>(p, cell_index<D>(own, g), sub, P1, val);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    if (mode[k] == 1) {
      val[1 + k] = -val[1 + k];
    } else if (mode[k] >= 2) {
      // 2 + 2 face: the inflow face's state; 14 + 2 face + part: a front part's
      const int m = mode[k] - 2;
      const double* q = (m < 12) ? g.bstate[m / 2] : g.front_state[(m - 12) / 2][(m - 12) % 2];
#pragma unroll
      for (int v = 0; v < NV; ++v) val[v] = q[v];
    }
  }
}

// L0: patch[j][v][L^d], local subcell -3..Ns+2 per axis around troubled cell
// list[chunk0 + j], ghosts by patch_value.
// Offset of local subcell loc (-3 .. Ns+2 per axis) in a limiter patch.
template <int D, int L>
__device__ __forceinline__ int patch_offset(const int* loc) {
  int off = 0, m = 1;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    off += (loc[k] + 3) * m;
    m *= L;
  }
  return off;
}

// Limiter patch of each troubled cell: v^n on L^D subcells (the cell and
// three layers around it, Eq. ader.icbc), each value as patch_value gives it
// and in the same operation order, gathered by neighbour boxes.  The patch
// splits into 3^D boxes, one per neighbour offset o in {-1, 0, 1}^D (per axis
// the 3 subcell layers below the cell, its Ns subcells, or the 3 layers
// above).  A box whose owner is one cell reached without a boundary ghost
// rule (an interior or periodic neighbour) is copied from that cell's stored
// subcell data when it was troubled at level n, else projected from its DOFs
// by tensor passes of P, axis by axis over the box (about n FMA per value and
// axis instead of n^D per value); other boxes take patch_value per subcell.
// One block per (troubled cell, box).
template <int D, int N>
__global__ void __launch_bounds__(128) k_lim_patch(Batch bt, int pass) {
  pass = lim_pass(bt, pass);
  using DM = Dims<D, N>;
  constexpr int n = DM::n, NV = DM::NV, ND = DM::ND, Ns = DM::Ns, NSD = DM::NSD, L = DM::L, LD = DM::LD;
  constexpr int NB = ipow(3, D), NR = ipow(n, D - 1);
  __shared__ double P1[Ns * n];
  __shared__ double Us[NV * ND];
  __shared__ double T1[NV * Ns * NR];                     // after the x pass
  __shared__ double T2[(D == 3) ? NV * Ns * Ns * n : 1];  // after the y pass (3D)
  for (int i = threadIdx.x; i < Ns * n; i += blockDim.x) P1[i] = bt.pps[0]->ops->P1[i];
  for (long long item = blockIdx.x; item < bt.pre[bt.n] * NB; item += gridDim.x) {
    __syncthreads();
    const long long t = item / NB;
    const int b = (int)(item - t * NB);
    const LimItem it = lim_item(bt, t);
    const Params& p = *bt.pps[it.s];
    const Geo& g = p.geo;
    const int j = it.j;
    const long long cell = p.b.list[1 - p.cur][pass * p.chunk + j];
    int ijk[3];
    cell_coords<D>(cell, g, ijk);
    int o[3] = {0, 0, 0}, lo[3] = {0, 0, 0}, R[3] = {1, 1, 1}, own[3] = {0, 0, 0};
    bool simple = true;
    {
      int bb = b;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        o[k] = bb % 3 - 1;
        bb /= 3;
        lo[k] = o[k] < 0 ? -3 : (o[k] == 0 ? 0 : Ns);
        R[k] = o[k] == 0 ? Ns : 3;
        int c = ijk[k] + o[k];
        if (c < 0 || c >= g.n[k]) {
          if (g.periodic[k]) c = (c + g.n[k]) % g.n[k];
          else simple = false;
        }
        own[k] = c;
      }
    }
    const int nbox = R[0] * R[1] * R[2];
    double* dst = p.b.patch + (size_t)j * NV * LD;
    if (!simple) {
      // a ghost rule applies along some axis: per subcell
      for (int e = threadIdx.x; e < nbox; e += blockDim.x) {
        int r = e, loc[3] = {0, 0, 0};
#pragma unroll
        for (int k = 0; k < D; ++k) {
          loc[k] = lo[k] + r % R[k];
          r /= R[k];
        }
        double val[NV];
        patch_value<D, N>(p, ijk, loc, P1, val);
        const int off = patch_offset<D, L>(loc);
#pragma unroll
        for (int v = 0; v < NV; ++v) dst[v * LD + off] = val[v];
      }
      continue;
    }
    const long long oc = cell_index<D>(own, g);
    if (p.b.beta[p.cur][oc]) {
      // the owner's subcell data of level n
      const double* st = p.b.store[p.cur] + (size_t)p.b.slot[p.cur][oc] * NV * NSD;
      for (int e = threadIdx.x; e < NV * nbox; e += blockDim.x) {
        const int v = e / nbox;
        int r = e - v * nbox, loc[3] = {0, 0, 0}, sidx = 0, m = 1;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          loc[k] = lo[k] + r % R[k];
          r /= R[k];
          sidx += (loc[k] - o[k] * Ns) * m;
          m *= Ns;
        }
        dst[v * LD + patch_offset<D, L>(loc)] = st[v * NSD + sidx];
      }
      continue;
    }
    // P(u^n) of the owner over the box, by tensor passes (x, y[, z])
    const double* U = p.b.U[p.cur] + oc * (NV * ND);
    for (int e = threadIdx.x; e < NV * ND; e += blockDim.x) Us[e] = U[e];
    __syncthreads();
    for (int e = threadIdx.x; e < NV * R[0] * NR; e += blockDim.x) {
      const int v = e / (R[0] * NR);
      const int r = e - v * (R[0] * NR);
      const int sx = r % R[0], rest = r / R[0];
      const double* px = P1 + (lo[0] + sx - o[0] * Ns) * n;
      const double* u = Us + v * ND + rest * n;
      double acc = 0.0;
#pragma unroll
      for (int a = 0; a < n; ++a) acc += px[a] * u[a];
      T1[(v * R[0] + sx) * NR + rest] = acc;
    }
    __syncthreads();
    if (D == 2) {
      for (int e = threadIdx.x; e < NV * R[0] * R[1]; e += blockDim.x) {
        const int v = e / (R[0] * R[1]);
        const int r = e - v * (R[0] * R[1]);
        const int sx = r % R[0], sy = r / R[0];
        const double* py = P1 + (lo[1] + sy - o[1] * Ns) * n;
        const double* t1 = T1 + (v * R[0] + sx) * NR;
        double accb = 0.0;
#pragma unroll
        for (int bb = 0; bb < n; ++bb) accb += py[bb] * t1[bb];
        const int loc[3] = {lo[0] + sx, lo[1] + sy, 0};
        dst[v * LD + patch_offset<D, L>(loc)] = 0.0 + accb;   // as 0 + 1 * accb in subcell_value
      }
    } else {
      for (int e = threadIdx.x; e < NV * R[0] * R[1] * n; e += blockDim.x) {
        const int v = e / (R[0] * R[1] * n);
        int r = e - v * (R[0] * R[1] * n);
        const int sx = r % R[0];
        r /= R[0];
        const int sy = r % R[1], c = r / R[1];
        const double* py = P1 + (lo[1] + sy - o[1] * Ns) * n;
        const double* t1 = T1 + (v * R[0] + sx) * NR + c * n;
        double accb = 0.0;
#pragma unroll
        for (int bb = 0; bb < n; ++bb) accb += py[bb] * t1[bb];
        T2[((v * R[0] + sx) * R[1] + sy) * n + c] = accb;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < NV * nbox; e += blockDim.x) {
        const int v = e / nbox;
        int r = e - v * nbox;
        const int sx = r % R[0];
        r /= R[0];
        const int sy = r % R[1], sz = r / R[1];
        const double* pz = P1 + (lo[2] + sz - o[2] * Ns) * n;
        const double* t2 = T2 + ((v * R[0] + sx) * R[1] + sy) * n;
        double acc = 0.0;
#pragma unroll
        for (int c = 0; c < n; ++c) acc += pz[c] * t2[c];
        const int loc[3] = {lo[0] + sx, lo[1] + sy, lo[2] + sz};
        dst[v * LD + patch_offset<D, L>(loc)] = acc;
      }
    }
  }
}


// 1D WENO3 on five consecutive subcell averages u[0..4] (target subcell u[2]):
// values of the reconstruction at the 3 GL nodes of the target subcell.
// Weights w_k = lambda_k / t_k, t_k = (sigma_k + eps)^8, normalised; with
// a_k = lambda_k prod_{j != k} t_j the normalised weights are a_k / sum a, so
// one division serves all outputs (the plain form is used if a product of
// two t_j could overflow).
__device__ __forceinline__ void weno3(const double* u, const Ops* __restrict__ o, double* out) {
  double t[3], p0[3], p1[3], p2[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double* C = o->C[k];
    const double c0 = C[0] * u[k] + C[1] * u[k + 1] + C[2] * u[k + 2];
    const double c1 = C[3] * u[k] + C[4] * u[k + 1] + C[5] * u[k + 2];
    const double c2 = C[6] * u[k] + C[7] * u[k + 1] + C[8] * u[k + 2];
    // sigma = int_0^1 (p')^2 + (p'')^2 = c1^2 + 2 c1 c2 + 16/3 c2^2
    const double sigma = c1 * (c1 + 2.0 * c2) + (16.0 / 3.0) * c2 * c2;
    double tk = sigma + WENO_EPS;
    tk = tk * tk;
    tk = tk * tk;
    t[k] = tk * tk;
    p0[k] = c0 + c1 * o->E[1] + c2 * o->E[2];
    p1[k] = c0 + c1 * o->E[4] + c2 * o->E[5];
    p2[k] = c0 + c1 * o->E[7] + c2 * o->E[8];
  }
  double a0, a1, a2;
  if (t[0] < 1e150 && t[1] < 1e150 && t[2] < 1e150) {
    a0 = t[1] * t[2];
    a1 = WENO_LAMBDA_C * (t[0] * t[2]);
    a2 = t[0] * t[1];
  } else {
    a0 = 1.0 / t[0];
    a1 = WENO_LAMBDA_C / t[1];
    a2 = 1.0 / t[2];
  }
  const double inv = 1.0 / (a0 + a1 + a2);
  out[0] = (a0 * p0[0] + a1 * p0[1] + a2 * p0[2]) * inv;
  out[1] = (a0 * p1[0] + a1 * p1[1] + a2 * p1[2]) * inv;
  out[2] = (a0 * p2[0] + a1 * p2[1] + a2 * p2[2]) * inv;
}

// FP32 form of weno3 (mixed precision).  (sigma_k + eps)^8 underflows in FP32
// for smooth data, so every t_k is divided by the smallest:
// t_k = ((sigma_min + eps) / (sigma_k + eps))^8 lies in [0, 1] and the weights
// lambda_k t_k / sum_j lambda_j t_j are those of weno3 (an underflow to 0 is
// the exact limit).  The nodal values come straight from the stencil
// averages (Wf = E C per stencil).
__device__ __forceinline__ void weno3f(const float* u, const Ops* __restrict__ o, float* out) {
  float sg[3], v[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float* C = o->Cf[k];
    const float c1 = C[0] * u[k] + C[1] * u[k + 1] + C[2] * u[k + 2];
    const float c2 = C[3] * u[k] + C[4] * u[k + 1] + C[5] * u[k + 2];
    sg[k] = c1 * (c1 + 2.0f * c2) + (16.0f / 3.0f) * c2 * c2 + (float)WENO_EPS;
    const float* W = o->Wf[k];
#pragma unroll
    for (int a = 0; a < 3; ++a) v[k][a] = W[a * 3] * u[k] + W[a * 3 + 1] * u[k + 1] + W[a * 3 + 2] * u[k + 2];
  }
  const float smin = fminf(sg[0], fminf(sg[1], sg[2]));
  float wt[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float r = smin / sg[k];
    r = r * r;
    r = r * r;
    wt[k] = r * r * (k == 1 ? (float)WENO_LAMBDA_C : 1.0f);
  }
  const float inv = 1.0f / (wt[0] + wt[1] + wt[2]);
#pragma unroll
  for (int a = 0; a < 3; ++a) out[a] = (wt[0] * v[0][a] + wt[1] * v[1][a] + wt[2] * v[2][a]) * inv;
}

// L1..L3: sweep along axis K.  Input extents (L or Ns+2 per axis) with NNIN
// nodal values per element; the output has extent Ns+2 along K and 3 NNIN
// nodes (the new nodal index is the slowest digit).
// T: the sweeps' precision (double; float for the mixed-precision FP32
// reconstruction); the patch (input of the x sweep) is always FP64.
template <int D, int N, int K, typename T>
__global__ void __launch_bounds__(256) k_lim_sweep(Batch bt, int pass) {
  using DM = Dims<D, N>;
  constexpr int NV = DM::NV, L = DM::L, NE = DM::NE;
  constexpr int I0 = (0 < K) ? NE : L, I1 = (1 < K) ? NE : L, I2 = (D < 3) ? 1 : ((2 < K) ? NE : L);
  constexpr int O0 = (0 <= K) ? NE : L, O1 = (1 <= K) ? NE : L, O2 = (D < 3) ? 1 : ((2 <= K) ? NE : L);
  constexpr int NNIN = ipow(3, K);
  constexpr int INSZ = I0 * I1 * I2 * NNIN;
  constexpr int OUTSZ = O0 * O1 * O2 * NNIN;          // elements, each producing 3 values
  constexpr int STRIDE = ((K == 0) ? 1 : (K == 1 ? I0 : I0 * I1)) * NNIN;
  const Ops* ops = bt.pps[0]->ops;
  for (long long eg = blockIdx.x * (long long)blockDim.x + threadIdx.x;
       eg < bt.pre[bt.n] * (NV * OUTSZ); eg += (long long)gridDim.x * blockDim.x) {
    const long long t = eg / (NV * OUTSZ);
    const LimItem it = lim_item(bt, t);
    const Params& p = *bt.pps[it.s];
    T* out = reinterpret_cast<T*>(p.b.sweep[K]);
    const long long e = eg - t * (NV * OUTSZ) + (long long)it.j * (NV * OUTSZ);
    const long long jv = e / OUTSZ;
    int r = (int)(e - jv * OUTSZ);
    const int node = r % NNIN;
    r /= NNIN;
    const int x0 = r % O0;
    r /= O0;
    const int x1 = r % O1;
    const int x2 = r / O1;
    // input element whose axis-K index equals the output's (stencil x_K .. x_K + 4)
    const int off = x0 + I0 * (x1 + I1 * x2);
    const size_t src_off = jv * INSZ + (size_t)off * NNIN + node;
    T u[5];
    if (K == 0) {
      const double* src = p.b.patch + src_off;
#pragma unroll
      for (int q = 0; q < 5; ++q) u[q] = (T)src[q * STRIDE];
    } else {
      const T* src = reinterpret_cast<const T*>(p.b.sweep[K > 0 ? K - 1 : 0]) + src_off;
#pragma unroll
      for (int q = 0; q < 5; ++q) u[q] = src[q * STRIDE];
    }
    T res[3];
    if constexpr (sizeof(T) == sizeof(double)) weno3(u, ops, res);
    else weno3f(u, ops, res);
    const int ooff = x0 + O0 * (x1 + O1 * x2);
    T* dst = out + jv * (size_t)OUTSZ * 3 + (size_t)ooff * NNIN * 3 + node;
#pragma unroll
    for (int a = 0; a < 3; ++a) dst[a * NNIN] = res[a];
  }
}

// L4: degree-2 space-time predictor (Eq. pde.nc.dg2 with 3 GL nodes per axis
// and in time, 3 Picard sweeps) on the subcells whose traces the sub-face
// fluxes use: the Ns^d interior subcells and the Ns^(d-1) ghost subcells
// facing each of the 2d cell faces.  In mixed precision the first two sweeps
// run in FP32 and the last in FP64.
constexpr int SUBS_PER_BLOCK_2D = 4;
constexpr int SUBS_PER_BLOCK_3D = 2;

// index in the (Ns+2)^d block (array index = local + 1) of the r-th subcell
// of the interior + face-ghost set
template <int D, int Ns>
__device__ __forceinline__ int cross_subcell(int r) {
  constexpr int NE = Ns + 2, NSD = ipow(Ns, D), NSF = ipow(Ns, D - 1);
  int c[3] = {0, 0, 0};
  if (r < NSD) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
      c[k] = r % Ns + 1;
      r /= Ns;
    }
  } else {
    r -= NSD;
    const int k = r / (2 * NSF);
    r -= k * 2 * NSF;
    const int side = r / NSF;
    int t = r - side * NSF;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      if (a == k) {
        c[a] = side ? Ns + 1 : 0;
      } else {
        c[a] = t % Ns + 1;
        t /= Ns;
      }
    }
  }
  return c[0] + NE * (c[1] + NE * c[2]);
}

// n32: sweeps (of 3) run in FP32 before the FP64 ones (MIXED only; the same
// for the whole launch, so every block takes the same barriers).
// QF: the whole predictor in FP32 (n32 = 3) from an FP32 reconstruction, the
// space-time nodal values stored in FP32 (qsub read as float by k_lim_flux).
template <int D, int N, bool MIXED, typename WT, bool QF>
__global__ void __launch_bounds__(256) k_lim_predict(Batch bt, int pass, int n32) {
  using DM = Dims<D, N>;
  constexpr int NV = DM::NV, NST3 = DM::NST3, ND3 = DM::ND3, NED = DM::NED, Ns = DM::Ns;
  constexpr int NCROSS = DM::NSD + 2 * D * DM::NSF;
  constexpr int SPB = (D == 2) ? SUBS_PER_BLOCK_2D : SUBS_PER_BLOCK_3D;
  constexpr int SPBF = MIXED ? SPB : 1;
  constexpr int SPBD = QF ? 1 : SPB;           // FP64 staging (unused when QF)
  __shared__ double su[SPBD][NV * ND3];
  __shared__ double sq[SPBD][NV * NST3];
  __shared__ double sF[SPBD][D * NV * NST3];
  __shared__ float suf[SPBF][NV * ND3];
  __shared__ float sqf[SPBF][NV * NST3];
  __shared__ float sFf[SPBF][D * NV * NST3];
  __shared__ double D3[9], K3[9];
  __shared__ float D3f[9], K3f[9];
  if (threadIdx.x < 9) {
    const Ops* o = bt.pps[0]->ops;
    D3[threadIdx.x] = o->D3[threadIdx.x];
    K3[threadIdx.x] = o->Kt3[threadIdx.x];
    D3f[threadIdx.x] = (float)o->D3[threadIdx.x];
    K3f[threadIdx.x] = (float)o->Kt3[threadIdx.x];
  }
  const int grp = threadIdx.x / NST3, lt = threadIdx.x - grp * NST3;
  const bool active_thread = grp < SPB;
  const long long total = bt.pre[bt.n] * NCROSS;
  for (long long base = (long long)blockIdx.x * SPB; base < total;
       base += (long long)gridDim.x * SPB) {
    const long long item = base + grp;
    const bool live = active_thread && item < total;
    const long long tg = live ? item / NCROSS : 0;
    const LimItem it = lim_item(bt, tg);
    const Params& p = *bt.pps[it.s];
    const long long j = it.j;
    const int sc = live ? cross_subcell<D, Ns>((int)(item - tg * NCROSS)) : 0;
    double c[3];
    float cf[3];
    {
#pragma unroll
      for (int k = 0; k < D; ++k) {
        c[k] = p.b.coef[3 + k];
        cf[k] = (float)c[k];
      }
    }
    const double gm1 = p.gamma - 1.0;
    const WT* W = reinterpret_cast<const WT*>(p.b.sweep[D - 1]);   // [j][v][NED][ND3]
    __syncthreads();
    if constexpr (QF) {
      if (live)
        for (int e = lt; e < NV * ND3; e += NST3) {
          const int v = e / ND3, i = e - v * ND3;
          suf[grp][e] = (float)W[((j * NV + v) * NED + sc) * ND3 + i];
        }
      __syncthreads();
      if (live)
        for (int e = lt; e < NV * NST3; e += NST3) {
          const int v = e / NST3, l = e - v * NST3;
          sqf[grp][e] = suf[grp][v * ND3 + (l % ND3)];
        }
      __syncthreads();
      for (int it = 0; it < 3; ++it) {
        if (live) picard_flux<D, 3, float>(sqf[grp], sFf[grp], (float)gm1, lt, NST3);
        __syncthreads();
        if (live) picard_deriv_sub<D>(sFf[grp], sqf[grp], cf, lt, NST3);
        __syncthreads();
        if (live) picard_time_sub<D>(sqf[grp], suf[grp], lt, NST3);
        __syncthreads();
      }
      if (live) {
        float* dst = reinterpret_cast<float*>(p.b.qsub) + ((size_t)j * NED + sc) * (size_t)(NV * NST3);
        for (int e = lt; e < NV * NST3; e += NST3) dst[e] = sqf[grp][e];
      }
      continue;
    }
    if (live) {
      for (int e = lt; e < NV * ND3; e += NST3) {
        const int v = e / ND3, i = e - v * ND3;
        su[grp][e] = (double)W[((j * NV + v) * NED + sc) * ND3 + i];
      }
    }
    __syncthreads();
    int it0 = 0;
    if (MIXED && n32 > 0) {
      if (live) {
        for (int e = lt; e < NV * ND3; e += NST3) suf[grp][e] = (float)su[grp][e];
        for (int e = lt; e < NV * NST3; e += NST3) {
          const int v = e / NST3, l = e - v * NST3;
          sqf[grp][e] = (float)su[grp][v * ND3 + (l % ND3)];
        }
      }
      __syncthreads();
      for (int it = 0; it < n32; ++it) {
        if (live) picard_flux<D, 3, float>(sqf[grp], sFf[grp], (float)gm1, lt, NST3);
        __syncthreads();
        if (live) picard_deriv<D, 3, float>(sFf[grp], sqf[grp], D3f, cf, lt, NST3);
        __syncthreads();
        if (live) picard_time<D, 3, float>(sqf[grp], suf[grp], K3f, lt, NST3);
        __syncthreads();
      }
      if (live)
        for (int e = lt; e < NV * NST3; e += NST3) sq[grp][e] = (double)sqf[grp][e];
      it0 = n32;
    } else if (live) {
      for (int e = lt; e < NV * NST3; e += NST3) {
        const int v = e / NST3, l = e - v * NST3;
        sq[grp][e] = su[grp][v * ND3 + (l % ND3)];
      }
    }
    __syncthreads();
    for (int it = it0; it < 3; ++it) {
      if (live) picard_flux<D, 3, double>(sq[grp], sF[grp], gm1, lt, NST3);
      __syncthreads();
      if (live) picard_deriv<D, 3, double>(sF[grp], sq[grp], D3, c, lt, NST3);
      __syncthreads();
      if (live) picard_time<D, 3, double>(sq[grp], su[grp], K3, lt, NST3);
      __syncthreads();
    }
    if (live) {
      double* dst = p.b.qsub + ((size_t)j * NED + sc) * (size_t)(NV * NST3);
      for (int e = lt; e < NV * NST3; e += NST3) dst[e] = sq[grp][e];
    }
  }
}

// L4 in mixed precision with the whole subcell predictor in FP32 (the default
// of the FP32 subcell scheme): one warp per subcell, W subcells per block,
// each warp synchronised by __syncwarp alone (the per-subcell arithmetic of
// k_lim_predict's QF path, none of its block barriers, and no thread group
// straddling two warps).  The blocks loop over the pass's subcells.
template <int D>
struct LimWarps {
  static constexpr int W = (D == 2) ? 8 : 4;     // subcells per block (static shared memory)
};

template <int D, int N>
__global__ void __launch_bounds__(32 * LimWarps<D>::W) k_lim_predict_w(Batch bt) {
  using DM = Dims<D, N>;
  constexpr int NV = DM::NV, NST3 = DM::NST3, ND3 = DM::ND3, NED = DM::NED, Ns = DM::Ns;
  constexpr int NCROSS = DM::NSD + 2 * D * DM::NSF;
  constexpr int W = LimWarps<D>::W;
  __shared__ float suf[W][NV * ND3];
  __shared__ float sqf[W][NV * NST3];
  __shared__ float sFf[W][D * NV * NST3];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float* u = suf[w];
  float* q = sqf[w];
  float* F = sFf[w];
  const long long total = bt.pre[bt.n] * NCROSS;
  for (long long item = (long long)blockIdx.x * W + w; item < total;
       item += (long long)gridDim.x * W) {
    const long long tg = item / NCROSS;
    const LimItem it = lim_item(bt, tg);
    const Params& p = *bt.pps[it.s];
    const long long j = it.j;
    const int sc = cross_subcell<D, Ns>((int)(item - tg * NCROSS));
    float cf[3];
#pragma unroll
    for (int k = 0; k < D; ++k) cf[k] = p.b.coef_f[3 + k];
    const float gm1 = p.b.coef_f[6];
    const float* Wr = reinterpret_cast<const float*>(p.b.sweep[D - 1]);   // [j][v][NED][ND3]
    for (int e = lane; e < NV * ND3; e += 32) {
      const int v = e / ND3, i = e - v * ND3;
      u[e] = Wr[((j * NV + v) * NED + sc) * ND3 + i];
    }
    __syncwarp();
    for (int e = lane; e < NV * NST3; e += 32) {
      const int v = e / NST3, l = e - v * NST3;
      q[e] = u[v * ND3 + (l % ND3)];
    }
    __syncwarp();
    for (int sweep = 0; sweep < 3; ++sweep) {
      picard_flux<D, 3, float>(q, F, gm1, lane, 32);
      __syncwarp();
      picard_deriv_sub<D>(F, q, cf, lane, 32);
      __syncwarp();
      picard_time_sub<D>(q, u, lane, 32);
      __syncwarp();
    }
    float* dst = reinterpret_cast<float*>(p.b.qsub) + ((size_t)j * NED + sc) * (size_t)(NV * NST3);
    for (int e = lane; e < NV * NST3; e += 32) dst[e] = q[e];
    __syncwarp();
  }
}

// Face traces of the 2D subcell predictor, the input of k_lim_flux_t2: for
// each troubled cell j, axis k, sub-face e normal to k (the enumeration of
// k_lim_flux) and side (0: the left subcell's trace at its high end, 1: the
// right subcell's at its low end), 9 points times 4 variables, the point
// t = (tangential node digit) + 3 (time node).
template <int N>
struct SubTraces2 {
  static constexpr int Ns = 2 * N + 1, NFK = (Ns + 1) * Ns, NP = 9;
  static constexpr long long per_cell = 2LL * NFK * 2 * 4 * NP;     // floats
  __host__ __device__ static constexpr long long offset(int k, int e, int side) {
    return ((long long)(k * NFK + e) * 2 + side) * 4 * NP;
  }
};

// The same subcell predictor in 2D in registers, three subcells per warp:
// lane l < 27 works on subcell l / 9 of the warp's three and holds its spatial
// node (a, b) = (l % 3, (l / 3) % 3) with the three time nodes.  The space
// derivatives take their three operands from the lanes on the node's line by
// warp shuffles; the time solve (Ktau) runs on the lane's own time nodes; the
// first sweep, from u (x) 1, forms the space term once for the three time
// nodes.  The operation order of every output is that of picard_flux /
// picard_deriv_sub / picard_time_sub.  TRACES: the subcell's traces on the
// sub-faces of the flux kernels (SubTraces2), each evaluated as k_lim_flux
// evaluates it from the nodal values, instead of the nodal values.
template <int N, bool TRACES>
__global__ void __launch_bounds__(256) k_lim_predict_s2(Batch bt) {
  using DM = Dims<2, N>;
  constexpr int NV = 4, NST3 = 27, ND3 = 9, NED = DM::NED, Ns = DM::Ns;
  constexpr int NCROSS = DM::NSD + 4 * DM::NSF;
  const int lane = threadIdx.x & 31;
  const int l = lane < 27 ? lane : 26;                  // idle lanes mirror lane 26
  const int g = l / 9, node = l - 9 * g;                 // subcell slot, spatial node
  const int a = node % 3, b = node / 3;
  float da[3], db[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    da[j] = c_D3f[a * 3 + j];
    db[j] = c_D3f[b * 3 + j];
  }
  const int sx = l - a, sy = l - 3 * b;                 // first lanes of this node's lines
  // the trace weights in FP32, converted once per thread
  float ph0[3], ph1[3];
  {
    const Ops* o = bt.pps[0]->ops;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      ph0[j] = (float)o->phi03[j];
      ph1[j] = (float)o->phi13[j];
    }
  }
  const int wpb = blockDim.x >> 5;
  const long long total = bt.pre[bt.n] * NCROSS;
  const long long groups = (total + 2) / 3;
  for (long long grp = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); grp < groups;
       grp += (long long)gridDim.x * wpb) {
    const long long item = grp * 3 + g;
    const bool live = item < total && lane < 27;
    const long long tg = item < total ? item / NCROSS : 0;
    const LimItem it = lim_item(bt, tg);
    const Params& p = *bt.pps[it.s];
    const long long j0 = it.j;
    const int sc = item < total ? cross_subcell<2, Ns>((int)(item - tg * NCROSS)) : 0;
    const float cx = p.b.coef_f[3], cy = p.b.coef_f[4];
    const float gm1 = p.b.coef_f[6];
    const float* Wr = reinterpret_cast<const float*>(p.b.sweep[1]);   // [j][v][NED][ND3]
    float u[NV], q[3][NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = item < total ? Wr[((j0 * NV + v) * NED + sc) * ND3 + node] : 1.0f;
    // S = cx D x F_x + cy D y F_y at this lane's node (picard_deriv_sub's order)
    auto space_term = [&](const float* Q, float* Sv) {
      float F[2][4];
      euler_fluxes<2, float>(Q, gm1, F);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        float s = 0.0f;
        {
          const float x0 = __shfl_sync(0xffffffffu, F[0][v], sx);
          const float x1 = __shfl_sync(0xffffffffu, F[0][v], sx + 1);
          const float x2 = __shfl_sync(0xffffffffu, F[0][v], sx + 2);
          float acc = 0.0f;
          acc += da[0] * x0;
          acc += da[1] * x1;
          acc += da[2] * x2;
          s += cx * acc;
        }
        {
          const float x0 = __shfl_sync(0xffffffffu, F[1][v], sy);
          const float x1 = __shfl_sync(0xffffffffu, F[1][v], sy + 3);
          const float x2 = __shfl_sync(0xffffffffu, F[1][v], sy + 6);
          float acc = 0.0f;
          acc += db[0] * x0;
          acc += db[1] * x1;
          acc += db[2] * x2;
          s += cy * acc;
        }
        Sv[v] = s;
      }
    };
#pragma unroll 1
    for (int sweep = 0; sweep < 3; ++sweep) {
      float S[3][NV];
      if (sweep == 0) {
        space_term(u, S[0]);
#pragma unroll
        for (int v = 0; v < NV; ++v) S[1][v] = S[2][v] = S[0][v];
      } else {
#pragma unroll
        for (int m = 0; m < 3; ++m) space_term(q[m], S[m]);
      }
#pragma unroll
      for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          float acc = 0.0f;
#pragma unroll
          for (int jj = 0; jj < 3; ++jj) acc += c_K3f[m * 3 + jj] * S[jj][v];
          q[m][v] = u[v] - acc;
        }
    }
    if constexpr (!TRACES) {
      if (live) {
        float* dst = reinterpret_cast<float*>(p.b.qsub) + ((size_t)j0 * NED + sc) * (size_t)(NV * NST3);
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
          for (int m = 0; m < 3; ++m) dst[v * NST3 + m * ND3 + node] = q[m][v];
      }
    } else {
      using TR = SubTraces2<N>;
      float* trc = reinterpret_cast<float*>(p.b.qsub) + (size_t)j0 * TR::per_cell;
      const int cc[2] = {sc % (Ns + 2), sc / (Ns + 2)};
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int o = 1 - k;                              // the tangential axis
        // (lanes of different subcells disagree here: every lane takes part in
        // the shuffles and only writes when its subcell has these faces)
        const bool faces = cc[o] >= 1 && cc[o] <= Ns;
        const int ak = k == 0 ? a : b;
        const int base = k == 0 ? sx : sy;
        const int stk = k == 0 ? 1 : 3;
        const int d = k == 0 ? b : a;                     // tangential digit
        const int ft = (faces ? cc[o] - 1 : 0) * (k == 0 ? Ns + 1 : 1);
        const int kmul = k == 0 ? 1 : Ns;
        const bool wr_hi = live && faces && ak == 2 && cc[k] <= Ns;
        const bool wr_lo = live && faces && ak == 0 && cc[k] >= 1;
        // (offsets clamped into the cell's block when the lane does not write)
        float* hi = trc + TR::offset(k, ft + (cc[k] <= Ns ? cc[k] : Ns) * kmul, 0);
        float* lo = trc + TR::offset(k, ft + (cc[k] >= 1 ? cc[k] - 1 : 0) * kmul, 1);
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll 2
          for (int v = 0; v < NV; ++v) {
            const float x0 = __shfl_sync(0xffffffffu, q[m][v], base);
            const float x1 = __shfl_sync(0xffffffffu, q[m][v], base + stk);
            const float x2 = __shfl_sync(0xffffffffu, q[m][v], base + 2 * stk);
            if (wr_hi) hi[v * 9 + d + 3 * m] = ph1[0] * x0 + ph1[1] * x1 + ph1[2] * x2;
            if (wr_lo) lo[v * 9 + d + 3 * m] = ph0[0] * x0 + ph0[1] * x1 + ph0[2] * x2;
          }
      }
    }
  }
}

// Sub-face fluxes normal to axis k from the face traces of k_lim_predict_s2
// (2D, FP32 subcell scheme, Rusanov): three sub-faces per warp, lane
// 9 f + t evaluating the flux at point t of sub-face f from two contiguous
// trace rows, then the GL-weighted sum over each sub-face's 9 points in point
// order, as k_lim_flux accumulates it.  The result is stored in FP64.
template <int N, int k>
__global__ void __launch_bounds__(256) k_lim_flux_t2(Batch bt, int pass) {
  pass = lim_pass(bt, pass);
  using TR = SubTraces2<N>;
  constexpr int NV = 4, Ns = TR::Ns, NFK = TR::NFK, NP = TR::NP;
  constexpr int WPB = 8;
  __shared__ float wts[NP];
  __shared__ float gsum[WPB][3][NV][NP + 1];
  const Ops* o = bt.pps[0]->ops;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x < NP) {
    // the point's weight, formed in k_lim_flux's order (tangential digit, then time)
    const int d = threadIdx.x % 3, mt = threadIdx.x / 3;
    float wt = 1.0f;
    wt *= (float)o->w3[d];
    wt *= (float)o->w3[mt];
    wts[threadIdx.x] = wt;
  }
  __syncthreads();
  const int fl = lane < 27 ? lane / 9 : 2, t = lane < 27 ? lane % 9 : 8;   // idle lanes mirror lane 26
  const long long total = bt.pre[bt.n] * NFK;
  const long long groups = (total + 2) / 3;
  for (long long grp = (long long)blockIdx.x * WPB + w; grp < groups; grp += (long long)gridDim.x * WPB) {
    const long long f = grp * 3 + fl;
    const bool live = f < total;
    const long long tg = live ? f / NFK : 0;
    const LimItem it = lim_item(bt, tg);
    const Params& p = *bt.pps[it.s];
    const long long j = it.j;
    const int e = live ? (int)(f - tg * NFK) : 0;
    const int fck = k == 0 ? e % (Ns + 1) : e / Ns;     // the face's index along k
    int wall = 0;
    const bool lo_wall = fck == 0 && p.geo.bc[2 * k] == ADG_BC_REFLECTIVE;
    const bool hi_wall = fck == Ns && p.geo.bc[2 * k + 1] == ADG_BC_REFLECTIVE;
    if (live && (lo_wall || hi_wall)) {
      const long long cell = p.b.list[1 - p.cur][pass * p.chunk + j];
      int ijk[3];
      cell_coords<2>(cell, p.geo, ijk);
      if (lo_wall && ijk[k] == 0) wall = -1;
      if (hi_wall && ijk[k] == p.geo.n[k] - 1) wall = 1;
    }
    float G[NV] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (live) {
      const float* tr = reinterpret_cast<const float*>(p.b.qsub) + (size_t)j * TR::per_cell;
      const float* tl = tr + TR::offset(k, e, 0);
      const float* trr = tr + TR::offset(k, e, 1);
      float QL[NV], QR[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        QL[v] = tl[v * NP + t];
        QR[v] = trr[v * NP + t];
      }
      if (wall < 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) QL[v] = QR[v];
        QL[1 + k] = -QR[1 + k];
      } else if (wall > 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) QR[v] = QL[v];
        QR[1 + k] = -QL[1 + k];
      }
      rusanov_f<2>(QL, QR, k, p.b.coef_f[7], G);
    }
    if (lane < 27) {
#pragma unroll
      for (int v = 0; v < NV; ++v) gsum[w][fl][v][t] = G[v];
    }
    __syncwarp();
    if (lane < 3 * NV) {
      const int ff = lane / NV, v = lane - ff * NV;
      const long long fo = grp * 3 + ff;
      if (fo < total) {
        const long long tgo = fo / NFK;
        const LimItem ito = lim_item(bt, tgo);
        const Params& po = *bt.pps[ito.s];
        const int eo = (int)(fo - tgo * NFK);
        float acc = 0.0f;
#pragma unroll
        for (int q = 0; q < NP; ++q) acc += wts[q] * gsum[w][ff][v][q];
        po.b.fsub[k][((size_t)ito.j * NV + v) * NFK + eo] = (double)acc;
      }
    }
    __syncwarp();
  }
}

// Face traces of the 3D subcell predictor, the input of k_lim_flux_t: for
// each troubled cell j, axis k, sub-face e normal to k (the enumeration of
// k_lim_flux: digits over the axes, Ns + 1 values along k and Ns along the
// others) and side (0: the trace of the left subcell at its high end, 1: of
// the right subcell at its low end), 27 points times NV variables, where the
// point t enumerates the node digits of the two tangential axes (lower axis
// fastest) and then the time node.
template <int N>
struct SubTraces {
  static constexpr int Ns = 2 * N + 1, NSF = Ns * Ns, NFK = (Ns + 1) * NSF, NP = 27;
  static constexpr long long per_cell = 3LL * NFK * 2 * 5 * NP;     // floats
  __host__ __device__ static constexpr long long offset(int k, int e, int side) {
    return ((long long)(k * NFK + e) * 2 + side) * 5 * NP;
  }
};

// The 3D subcell predictor in registers: lane l < 27 holds spatial node
// (a, b, c) = (l % 3, (l / 3) % 3, l / 9) of the subcell and its three time
// nodes.  The space derivatives take their three operands per axis from the
// lanes on the node's line by warp shuffles; the time contraction
// (Ktau) runs on the lane's own three time nodes, so it needs no exchange at
// all, and the first sweep, from the time-constant u (x) 1, forms the space
// term once for the three time nodes.  A
// sweep uses no shared memory and no synchronisation.  The operation order of
// every output is that of picard_flux / picard_deriv_sub / picard_time_sub.
// The subcell's traces on the sub-faces the flux kernels use are written in
// place of its nodal values (SubTraces), each evaluated as k_lim_flux
// evaluates it from the nodal values.
template <int N>
__global__ void __launch_bounds__(256) k_lim_predict_s3(Batch bt) {
  using DM = Dims<3, N>;
  constexpr int NV = 5, NST3 = 81, ND3 = 27, NED = DM::NED, Ns = DM::Ns;
  constexpr int NCROSS = DM::NSD + 6 * DM::NSF;
  const int lane = threadIdx.x & 31;
  const int l = lane < ND3 ? lane : ND3 - 1;            // idle lanes mirror node 26
  const int a = l % 3, b = (l / 3) % 3, c = l / 9;
  float da[3], db[3], dc[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    da[j] = c_D3f[a * 3 + j];
    db[j] = c_D3f[b * 3 + j];
    dc[j] = c_D3f[c * 3 + j];
  }
  const int sx = l - a, sy = l - 3 * b, sz = l - 9 * c;   // first lanes of this node's lines
  // the trace weights in FP32, converted once per thread (FP64 -> FP32
  // conversions run on the narrow FP64 pipe)
  float ph0[3], ph1[3];
  {
    const Ops* o = bt.pps[0]->ops;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      ph0[j] = (float)o->phi03[j];
      ph1[j] = (float)o->phi13[j];
    }
  }
  const int wpb = blockDim.x >> 5;
  const long long total = bt.pre[bt.n] * NCROSS;
  for (long long item = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); item < total;
       item += (long long)gridDim.x * wpb) {
    const long long tg = item / NCROSS;
    const LimItem it = lim_item(bt, tg);
    const Params& p = *bt.pps[it.s];
    const long long j0 = it.j;
    const int sc = cross_subcell<3, Ns>((int)(item - tg * NCROSS));
    const float cf[3] = {p.b.coef_f[3], p.b.coef_f[4], p.b.coef_f[5]};
    const float gm1 = p.b.coef_f[6];
    const float* Wr = reinterpret_cast<const float*>(p.b.sweep[2]);   // [j][v][NED][ND3]
    float u[NV], q[3][NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      u[v] = Wr[((j0 * NV + v) * NED + sc) * ND3 + l];
#pragma unroll
      for (int m = 0; m < 3; ++m) q[m][v] = u[v];
    }
    // S = sum_k c_k D x_k f_k(Q) at this lane's node, in picard_deriv_sub's order
    auto space_term = [&](const float* Q, float* Sv) {
      float F[3][5];
      euler_fluxes<3, float>(Q, gm1, F);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int base = k == 0 ? sx : (k == 1 ? sy : sz);
          const int st = k == 0 ? 1 : (k == 1 ? 3 : 9);
          const float* dr = k == 0 ? da : (k == 1 ? db : dc);
          const float x0 = __shfl_sync(0xffffffffu, F[k][v], base);
          const float x1 = __shfl_sync(0xffffffffu, F[k][v], base + st);
          const float x2 = __shfl_sync(0xffffffffu, F[k][v], base + 2 * st);
          float acc = 0.0f;
          acc += dr[0] * x0;
          acc += dr[1] * x1;
          acc += dr[2] * x2;
          s += cf[k] * acc;
        }
        Sv[v] = s;
      }
    };
#pragma unroll 1
    for (int sweep = 0; sweep < 3; ++sweep) {
      float S[3][NV];
      if (sweep == 0) {
        // the first sweep starts from u (x) 1: its three time nodes carry the
        // same values, hence the same space term
        space_term(u, S[0]);
#pragma unroll
        for (int v = 0; v < NV; ++v) S[1][v] = S[2][v] = S[0][v];
      } else {
#pragma unroll
        for (int m = 0; m < 3; ++m) space_term(q[m], S[m]);
      }
#pragma unroll
      for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          float acc = 0.0f;
#pragma unroll
          for (int j = 0; j < 3; ++j) acc += c_K3f[m * 3 + j] * S[j][v];
          q[m][v] = u[v] - acc;
        }
    }
    // traces: the subcell's block coordinates (local + 1, 0 .. Ns + 1 per axis)
    using TR = SubTraces<N>;
    float* trc = reinterpret_cast<float*>(p.b.qsub) + (size_t)j0 * TR::per_cell;
    const int cc[3] = {sc % (Ns + 2), (sc / (Ns + 2)) % (Ns + 2), sc / ((Ns + 2) * (Ns + 2))};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      // a subcell has faces normal to k in the set when its other coordinates are interior
      bool inner = true;
#pragma unroll
      for (int x = 0; x < 3; ++x)
        if (x != k && (cc[x] < 1 || cc[x] > Ns)) inner = false;
      if (!inner) continue;                                 // uniform over the warp
      const int ak = k == 0 ? a : (k == 1 ? b : c);
      const int base = k == 0 ? sx : (k == 1 ? sy : sz);
      const int st = k == 0 ? 1 : (k == 1 ? 3 : 9);
      // tangential digits (lower axis first) and the face's tangential index
      const int d0 = k == 0 ? b : a, d1 = k == 2 ? b : c;
      int ft = 0, mul = 1;
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        const int ext = (x == k) ? Ns + 1 : Ns;
        if (x != k) ft += (cc[x] - 1) * mul;
        mul *= ext;
      }
      const int kmul = k == 0 ? 1 : (k == 1 ? Ns : Ns * Ns);   // place of fc[k] in e
      // left of face cc[k] (high-end trace, lanes with a_k = 2), right of
      // face cc[k] - 1 (low-end trace, lanes with a_k = 0)
      const bool wr_hi = ak == 2 && cc[k] <= Ns && lane < ND3;
      const bool wr_lo = ak == 0 && cc[k] >= 1 && lane < ND3;
      float* hi = trc + TR::offset(k, ft + cc[k] * kmul, 0);
      float* lo = trc + TR::offset(k, ft + (cc[k] - 1) * kmul, 1);
#pragma unroll
      for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const float x0 = __shfl_sync(0xffffffffu, q[m][v], base);
          const float x1 = __shfl_sync(0xffffffffu, q[m][v], base + st);
          const float x2 = __shfl_sync(0xffffffffu, q[m][v], base + 2 * st);
          const int t = d0 + 3 * d1 + 9 * m;
          if (wr_hi) hi[v * 27 + t] = ph1[0] * x0 + ph1[1] * x1 + ph1[2] * x2;
          if (wr_lo) lo[v * 27 + t] = ph0[0] * x0 + ph0[1] * x1 + ph0[2] * x2;
        }
    }
  }
}

// Sub-face fluxes normal to axis k from the face traces of k_lim_predict_s3
// (3D, FP32 subcell scheme, Rusanov): one warp per sub-face, lane t < 27
// evaluates the flux at point t of the face (its two traces are contiguous
// across the lanes), then the GL-weighted sum over the 27 points runs in
// point order, as k_lim_flux accumulates it.  The result is stored in FP64.
template <int N, int k>
__global__ void __launch_bounds__(256) k_lim_flux_t(Batch bt, int pass) {
  pass = lim_pass(bt, pass);
  using TR = SubTraces<N>;
  constexpr int NV = 5, Ns = TR::Ns, NFK = TR::NFK, NP = TR::NP;
  constexpr int WPB = 8;
  __shared__ float wts[NP];
  __shared__ float gsum[WPB][NV][NP + 1];
  const Ops* o = bt.pps[0]->ops;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x < NP) {
    // the point's weight, formed in k_lim_flux's order
    int tt = threadIdx.x;
    float wt = 1.0f;
#pragma unroll
    for (int x = 0; x < 3; ++x)
      if (x != k) {
        wt *= (float)o->w3[tt % 3];
        tt /= 3;
      }
    wt *= (float)o->w3[tt];
    wts[threadIdx.x] = wt;
  }
  __syncthreads();
  const int t = lane < NP ? lane : NP - 1;                 // idle lanes mirror point 26
  const long long total = bt.pre[bt.n] * NFK;
  for (long long item = (long long)blockIdx.x * WPB + w; item < total;
       item += (long long)gridDim.x * WPB) {
    const long long tg = item / NFK;
    const LimItem it = lim_item(bt, tg);
    const Params& p = *bt.pps[it.s];
    const long long j = it.j;
    const int e = (int)(item - tg * NFK);
    // the face's index along k (e = fc0 + ext0 (fc1 + ext1 fc2))
    const int fck = k == 0 ? e % (Ns + 1) : (k == 1 ? (e / Ns) % (Ns + 1) : e / (Ns * Ns));
    // reflecting walls: as in k_lim_flux
    int wall = 0;
    const bool lo_wall = fck == 0 && p.geo.bc[2 * k] == ADG_BC_REFLECTIVE;
    const bool hi_wall = fck == Ns && p.geo.bc[2 * k + 1] == ADG_BC_REFLECTIVE;
    if (lo_wall || hi_wall) {
      const long long cell = p.b.list[1 - p.cur][pass * p.chunk + j];
      int ijk[3];
      cell_coords<3>(cell, p.geo, ijk);
      if (lo_wall && ijk[k] == 0) wall = -1;
      if (hi_wall && ijk[k] == p.geo.n[k] - 1) wall = 1;
    }
    const float* tr = reinterpret_cast<const float*>(p.b.qsub) + (size_t)j * TR::per_cell;
    const float* tl = tr + TR::offset(k, e, 0);
    const float* trr = tr + TR::offset(k, e, 1);
    float QL[NV], QR[NV], G[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      QL[v] = tl[v * NP + t];
      QR[v] = trr[v * NP + t];
    }
    if (wall < 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) QL[v] = QR[v];
      QL[1 + k] = -QR[1 + k];
    } else if (wall > 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) QR[v] = QL[v];
      QR[1 + k] = -QL[1 + k];
    }
    rusanov_f<3>(QL, QR, k, p.b.coef_f[7], G);
    if (lane < NP) {
#pragma unroll
      for (int v = 0; v < NV; ++v) gsum[w][v][lane] = G[v];
    }
    __syncwarp();
    if (lane < NV) {
      float acc = 0.0f;
#pragma unroll
      for (int q = 0; q < NP; ++q) acc += wts[q] * gsum[w][lane][q];
      p.b.fsub[k][((size_t)j * NV + lane) * NFK + e] = (double)acc;
    }
    __syncwarp();
  }
}

// L5: sub-face fluxes normal to axis k: Rusanov at the 3^(d-1) x 3
// tangential x time GL points, averaged with the GL weights.  Faces f = 0..Ns
// along k (between local subcells f-1 and f), tangential subcells 0..Ns-1.
// T: the flux precision (double; float for the mixed-precision FP32 subcell
// scheme, Rusanov only); the result is stored in FP64.
// QT: the element type of the stored subcell predictor (float when it ran
// wholly in FP32, see k_lim_predict).
template <int D, int N, int k, typename T, typename QT>
__global__ void __launch_bounds__(256) k_lim_flux(Batch bt, int pass) {
  pass = lim_pass(bt, pass);
  using DM = Dims<D, N>;
  constexpr int NV = DM::NV, NST3 = DM::NST3, ND3 = DM::ND3, NE = DM::NE, NED = DM::NED,
                Ns = DM::Ns;
  constexpr int NFK = (Ns + 1) * DM::NSF;
  const Ops* o = bt.pps[0]->ops;
  constexpr int stk = (k == 0) ? 1 : (k == 1 ? 3 : 9);   // node stride of axis k
  // the GL weights and trace weights in T, converted once per thread
  T w3t[3], p0t[3], p1t[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    w3t[q] = (T)o->w3[q];
    p0t[q] = (T)o->phi03[q];
    p1t[q] = (T)o->phi13[q];
  }
  for (long long eg = blockIdx.x * (long long)blockDim.x + threadIdx.x; eg < bt.pre[bt.n] * NFK;
       eg += (long long)gridDim.x * blockDim.x) {
    const long long tg = eg / NFK;
    const LimItem it = lim_item(bt, tg);
    const Params& p = *bt.pps[it.s];
    const long long j = it.j;
    const long long e = j * NFK + (eg - tg * NFK);
    int r = (int)(e - j * NFK);
    int fc[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int ext = (a == k) ? Ns + 1 : Ns;
      fc[a] = r % ext;
      r /= ext;
    }
    // left / right subcells in the (Ns+2)^d block (array index = local + 1)
    int sl = 0, sr = 0, mul = 1;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int il = (a == k) ? fc[a] : fc[a] + 1;
      const int ir = (a == k) ? fc[a] + 1 : fc[a] + 1;
      sl += il * mul;
      sr += ir * mul;
      mul *= NE;
    }
    const QT* qL = reinterpret_cast<const QT*>(p.b.qsub) + ((size_t)j * NED + sl) * NV * NST3;
    const QT* qR = reinterpret_cast<const QT*>(p.b.qsub) + ((size_t)j * NED + sr) * NV * NST3;
    // a sub-face on a reflecting wall takes its flux between the interior
    // trace and its mirror image (no mass or energy through the wall)
    // (the troubled-cell list is read only when the face can be a wall: the
    // no-allocation entry point runs this kernel with periodic kinds and no list)
    int wall = 0;                          // -1: low wall (ghost left), +1: high wall (ghost right)
    const bool lo_wall = fc[k] == 0 && p.geo.bc[2 * k] == ADG_BC_REFLECTIVE;
    const bool hi_wall = fc[k] == Ns && p.geo.bc[2 * k + 1] == ADG_BC_REFLECTIVE;
    if (lo_wall || hi_wall) {
      const long long cell = p.b.list[1 - p.cur][pass * p.chunk + j];
      int ijk[3];
      cell_coords<D>(cell, p.geo, ijk);
      if (lo_wall && ijk[k] == 0) wall = -1;
      if (hi_wall && ijk[k] == p.geo.n[k] - 1) wall = 1;
    }
    T acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = T(0);
    const float gf = p.b.coef_f ? p.b.coef_f[7] : (float)p.gamma;
    // tangential x time nodes: digits over axes != k, then time
    for (int t = 0; t < ND3; ++t) {
      int base = 0, tt = t, wmul = 1;
      T wt = T(1);
      int st = 1;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        if (a != k) {
          const int dg = tt % 3;
          tt /= 3;
          base += dg * st;
          wt *= dg == 0 ? w3t[0] : (dg == 1 ? w3t[1] : w3t[2]);   // (registers, not a local array)
        }
        st *= 3;
      }
      const int m = tt;                 // remaining digit: time node
      wt *= m == 0 ? w3t[0] : (m == 1 ? w3t[1] : w3t[2]);
      base += m * ND3;
      (void)wmul;
      T QL[NV], QR[NV], G[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const QT* a = qL + v * NST3 + base;
        const QT* b = qR + v * NST3 + base;
        QL[v] = p1t[0] * (T)a[0] + p1t[1] * (T)a[stk] + p1t[2] * (T)a[2 * stk];
        QR[v] = p0t[0] * (T)b[0] + p0t[1] * (T)b[stk] + p0t[2] * (T)b[2 * stk];
      }
      if (wall < 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) QL[v] = QR[v];
        QL[1 + k] = -QR[1 + k];
      } else if (wall > 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) QR[v] = QL[v];
        QR[1 + k] = -QL[1 + k];
      }
      if constexpr (sizeof(T) == sizeof(double)) face_flux<D>(p.flux, QL, QR, k, p.gamma, G);
      else rusanov_f<D>(QL, QR, k, gf, G);
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] += wt * G[v];
    }
    double* dst = p.b.fsub[k] + (size_t)j * NV * NFK + (e - j * NFK);
#pragma unroll
    for (int v = 0; v < NV; ++v) dst[v * NFK] = (double)acc[v];
  }
}

// L6: finite volume update, storage of v^{n+1}, reconstruction R, per-cell
// min/max and wave speed, sub-face fluxes of the cell faces, and marking of
// unlimited face neighbours for the flux correction.  One block per cell.
template <int D, int N>
__global__ void __launch_bounds__(128) k_lim_update(Batch bt, int pass) {
  pass = lim_pass(bt, pass);
  using DM = Dims<D, N>;
  constexpr int n = DM::n, NV = DM::NV, ND = DM::ND, Ns = DM::Ns, NSD = DM::NSD, L = DM::L,
                LD = DM::LD, NSF = DM::NSF;
  constexpr int NFK = (Ns + 1) * NSF;
  extern __shared__ double sm[];
  double* A = sm;                 // NV * NSD
  double* B = A + NV * NSD;       // NV * NSD
  double* R1 = B + NV * NSD;      // n * Ns
  double* mm = R1 + n * Ns;       // 2 NV
  double* red = mm + 2 * NV;      // 128
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int i = tid; i < n * Ns; i += nth) R1[i] = bt.pps[0]->ops->R1[i];
  for (long long tg = blockIdx.x; tg < bt.pre[bt.n]; tg += gridDim.x) {
    const LimItem it = lim_item(bt, tg);
    const Params& p = *bt.pps[it.s];
    const int j = it.j;
    const int nxt = 1 - p.cur;
    double c[3];
    {
#pragma unroll
      for (int k = 0; k < D; ++k) c[k] = p.b.coef[3 + k];
    }
    const int t = pass * p.chunk + j;
    const long long cell = p.b.list[nxt][t];
    const double* pt = p.b.patch + (size_t)j * NV * LD;
    double* st = p.b.store[nxt] + (size_t)t * NV * NSD;
    __syncthreads();
    for (int e = tid; e < NV * NSD; e += nth) {
      const int v = e / NSD;
      int s = e - v * NSD;
      int sc[3] = {0, 0, 0};
#pragma unroll
      for (int a = 0; a < D; ++a) {
        sc[a] = s % Ns;
        s /= Ns;
      }
      int poff = 0, pm = 1;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        poff += (sc[a] + 3) * pm;
        pm *= L;
      }
      double val = pt[v * LD + poff];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        int flo = 0, mul = 1;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          flo += sc[a] * mul;
          mul *= (a == k) ? Ns + 1 : Ns;
        }
        const int kst = (k == 0) ? 1 : (k == 1 ? Ns : Ns * Ns);   // stride of axis k
        const double* F = p.b.fsub[k] + ((size_t)j * NV + v) * NFK;
        val -= c[k] * (F[flo + kst] - F[flo]);
      }
      A[e] = val;
      st[e] = val;
    }
    __syncthreads();
    double lam = 0.0;
    const bool bad = check_subcells<D>(A, NSD, nullptr, p.gamma, mm, p.lam_mode ? &lam : nullptr, red,
                                       p.prec == ADG_PREC_MIXED_FP32, p.gam2f);
    if (tid == 0) {
      if (p.lam_mode) p.b.lam[cell] = lam;
      if (bad && p.cascade) {
        // first-order layer: recomputed by k_lim_fallback after all passes
        const int i = atomicAdd(&p.b.counters[CNT_FB], 1);
        p.b.fblist[i] = t;
        p.b.fbflag[t] = p.stamp;
        atomicAdd(&p.b.counters[CNT_FB_TOTAL], 1);
      } else if (bad) {
        atomicAdd(&p.b.counters[CNT_INADM], 1);
      }
    }
    if (tid < 2 * NV) p.b.cmm[nxt][cell * 2 * NV + tid] = mm[tid];
    // sub-face fluxes on the faces of the cell: edge[t][k][side][v][NSF]
    for (int e = tid; e < D * 2 * NV * NSF; e += nth) {
      const int k = e / (2 * NV * NSF);
      int r = e - k * (2 * NV * NSF);
      const int side = r / (NV * NSF);
      r -= side * NV * NSF;
      const int v = r / NSF, ts = r - v * NSF;
      int tc[2] = {ts % Ns, ts / Ns};
      int fidx = 0, mul = 1, q = 0;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int cc = (a == k) ? (side ? Ns : 0) : tc[q++];
        fidx += cc * mul;
        mul *= (a == k) ? Ns + 1 : Ns;
      }
      p.b.edge[(size_t)t * D * 2 * NV * NSF + e] = p.b.fsub[k][((size_t)j * NV + v) * NFK + fidx];
    }
    // reconstruction R of the new subcell data
    __syncthreads();
    double* u = apply_ct<D, NV, Ns, n>(A, B, R1, tid, nth);
    double* Uo = p.b.U[nxt] + cell * (NV * ND);
    for (int e = tid; e < NV * ND; e += nth) Uo[e] = u[e];
    if (tid == 0 && p.b.vok) p.b.vok[cell] = 0;     // P(R(v)) is not v: recompute next step
    // unlimited face neighbours get the flux correction
    if (tid < 2 * D) {
      const int k = tid >> 1, side = (tid & 1) ? 1 : -1;
      int ijk[3], nb[3];
      cell_coords<D>(cell, p.geo, ijk);
      if (face_neighbour<D>(p.geo, ijk, k, side, nb)) {
        const long long nc = cell_index<D>(nb, p.geo);
        if (!p.b.beta[nxt][nc]) {
          const int old = atomicExch(&p.b.fixstamp[nc], p.stamp);
          if (old != p.stamp) {
            const int idx = atomicAdd(&p.b.counters[CNT_FIX], 1);
            p.b.fixlist[idx] = (int)nc;
          }
        }
      }
    }
  }
}

// L7: flux correction of unlimited cells with troubled face neighbours
// (Sec. 4.4): on each such face the DG flux Gbar is replaced by the sub-face
// fluxes integrated against the test functions,
//   Fsub_b = (1/W_b) sum_e Fbar_e prod P1[e][b] / Ns^(d-1).
template <int D, int N>
__global__ void __launch_bounds__(128) k_lim_fix(Batch bt) {
  using DM = Dims<D, N>;
  constexpr int n = DM::n, NV = DM::NV, ND = DM::ND, NF = DM::NF, Ns = DM::Ns, NSD = DM::NSD,
                NSF = DM::NSF;
  extern __shared__ double sm[];
  double* U = sm;                      // NV * ND
  double* A = U + NV * ND;             // NV * max(NSD, ...)
  double* B = A + NV * NSD;
  double* Mt = B + NV * NSD;           // n * Ns
  double* P1 = Mt + n * Ns;            // Ns * n
  double* mm = P1 + Ns * n;
  double* red = mm + 2 * NV;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int i = tid; i < n * Ns; i += nth) {
    Mt[i] = bt.pps[0]->ops->Mt[i];
    P1[i] = bt.pps[0]->ops->P1[i];
  }
  for (long long fg = blockIdx.x; fg < bt.pre[bt.n]; fg += gridDim.x) {
    const int sidx = batch_state(bt, fg);
    const Params& p = *bt.pps[sidx];
    const long long f = fg - bt.pre[sidx];
    const int nxt = 1 - p.cur;
    const long long cell = p.b.fixlist[f];
    int ijk[3];
    cell_coords<D>(cell, p.geo, ijk);
    double* Uo = p.b.U[nxt] + cell * (NV * ND);
    __syncthreads();
    for (int e = tid; e < NV * ND; e += nth) U[e] = Uo[e];
    for (int k = 0; k < D; ++k) {
      const double ck = p.b.coef[k];
      for (int side = -1; side <= 1; side += 2) {
        int nb[3];
        if (!face_neighbour<D>(p.geo, ijk, k, side, nb)) continue;
        const long long nc = cell_index<D>(nb, p.geo);
        if (!p.b.beta[nxt][nc]) continue;
        const int slot = p.b.slot[nxt][nc];
        if (slot < 0) continue;
        // the neighbour's face that touches this cell
        const int eside = (side > 0) ? 0 : 1;
        const double* Fs = p.b.edge + (size_t)slot * D * 2 * NV * NSF + ((size_t)k * 2 + eside) * NV * NSF;
        __syncthreads();
        // project the Ns^(d-1) sub-face fluxes on the n^(d-1) tangential nodes
        for (int e = tid; e < NV * NSF; e += nth) A[e] = Fs[e];
        __syncthreads();
        double* Fp = A;
        if (D == 2) {
          int ext[3] = {Ns, 1, 1};
          apply_axis<1>(A, B, Mt, n, Ns, 0, ext, NV, tid, nth);
          Fp = B;
        } else {
          int ext[3] = {Ns, Ns, 1};
          apply_axis<2>(A, B, Mt, n, Ns, 0, ext, NV, tid, nth);
          __syncthreads();
          ext[0] = n;
          apply_axis<2>(B, A, Mt, n, Ns, 1, ext, NV, tid, nth);
          Fp = A;
        }
        __syncthreads();
        const long long face = face_index<D>(p.geo, ijk, k, side > 0 ? ijk[k] + 1 : ijk[k]);
        const double* Gd = p.b.G[k] + face * NV * NF;
        for (int e = tid; e < NV * ND; e += nth) {
          const int v = e / ND, i = e - v * ND;
          const int st = (k == 0) ? 1 : (k == 1 ? n : n * n);
          const int ak = (i / st) % n;
          const int ts = tangential<D, n>(i, k);
          const double diff = Fp[v * NF + ts] - Gd[v * NF + ts];
          if (side > 0) U[e] -= ck * p.ops->phi1w[ak] * diff;
          else U[e] += ck * p.ops->phi0w[ak] * diff;
        }
      }
    }
    __syncthreads();
    for (int e = tid; e < NV * ND; e += nth) {
      Uo[e] = U[e];
      A[e] = U[e];
    }
    __syncthreads();
    double* vs = apply_ct<D, NV, n, Ns>(A, B, P1, tid, nth);
    if (p.b.vstar) {
      // the corrected DOFs' projection, kept for the next step's detector
      double* vk = p.b.vstar + cell * (size_t)(NV * NSD);
      for (int e = tid; e < NV * NSD; e += nth) vk[e] = vs[e];
    }
    double lam = 0.0;
    check_subcells<D>(vs, NSD, nullptr, p.gamma, mm, p.lam_mode ? &lam : nullptr, red,
                      p.prec == ADG_PREC_MIXED_FP32, p.gam2f);
    if (tid == 0 && p.lam_mode) p.b.lam[cell] = lam;
    if (tid < 2 * NV) p.b.cmm[nxt][cell * 2 * NV + tid] = mm[tid];
  }
}

// Cascade layer (Sec. 6, Fig. algo2), part 1: each troubled cell whose WENO3
// result failed PAD is recomputed from v^n by one first-order Rusanov step on
// its subgrid: sub-face fluxes between the piecewise-constant subcell data,
// ghost data from Eq. (ader.icbc) as for the WENO3 patch (wrapped or clamped
// global subcell index).  Writes v^{n+1}, min / max, wave speed, u = R(v) and
// the cell-face fluxes (the flux correction of unlimited neighbours uses
// them), and lists the WENO3 face neighbours, which must take the
// first-order flux on the shared face (part 2).  One block per cell.
template <int D, int N>
__global__ void __launch_bounds__(128) k_lim_fallback(Batch bt) {
  using DM = Dims<D, N>;
  constexpr int n = DM::n, NV = DM::NV, ND = DM::ND, Ns = DM::Ns, NSD = DM::NSD, NSF = DM::NSF;
  constexpr int NE = Ns + 2;                          // local subcells -1..Ns per axis
  constexpr int NB = (D == 3) ? NE * NE * NE : NE * NE;
  constexpr int NFK = (Ns + 1) * NSF;
  extern __shared__ double sm[];
  double* blk = sm;                 // NV * NB   v^n with one ghost layer
  double* A = blk + NV * NB;        // NV * NSD
  double* B = A + NV * NSD;         // NV * NSD
  double* F = B + NV * NSD;         // NV * NFK  sub-face fluxes of one axis
  double* R1 = F + NV * NFK;        // n * Ns
  double* P1 = R1 + n * Ns;         // Ns * n
  double* mm = P1 + Ns * n;         // 2 NV
  double* red = mm + 2 * NV;        // 128
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int i = tid; i < n * Ns; i += nth) {
    R1[i] = bt.pps[0]->ops->R1[i];
    P1[i] = bt.pps[0]->ops->P1[i];
  }
  for (long long fg = blockIdx.x; fg < bt.pre[bt.n]; fg += gridDim.x) {
    const int sidx = batch_state(bt, fg);
    const Params& p = *bt.pps[sidx];
    const long long f = fg - bt.pre[sidx];
    const int nxt = 1 - p.cur;
    const Geo& g = p.geo;
    const int t = p.b.fblist[f];
    const long long cell = p.b.list[nxt][t];
    int ijk[3];
    cell_coords<D>(cell, g, ijk);
    __syncthreads();
    for (int e = tid; e < NB; e += nth) {
      int r = e;
      int loc[3] = {0, 0, 0};
#pragma unroll
      for (int k = 0; k < D; ++k) {
        loc[k] = r % NE - 1;
        r /= NE;
      }
      double val[NV];
      patch_value<D, N>(p, ijk, loc, P1, val);
#pragma unroll
      for (int v = 0; v < NV; ++v) blk[v * NB + e] = val[v];
    }
    __syncthreads();
    for (int e = tid; e < NV * NSD; e += nth) {
      const int v = e / NSD;
      int s = e - v * NSD, bi = 0, mul = 1;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        bi += (s % Ns + 1) * mul;
        s /= Ns;
        mul *= NE;
      }
      A[e] = blk[v * NB + bi];
    }
    for (int k = 0; k < D; ++k) {
      const double ck = p.b.coef[3 + k];
      __syncthreads();
      // faces c_k = 0..Ns between local subcells c_k - 1 and c_k
      for (int e = tid; e < NFK; e += nth) {
        int r = e, bl = 0, mul = 1, stk = 1;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const int ext = (a == k) ? Ns + 1 : Ns;
          const int c = r % ext;
          r /= ext;
          bl += (a == k ? c : c + 1) * mul;
          if (a == k) stk = mul;
          mul *= NE;
        }
        double QL[NV], QR[NV], G[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          QL[v] = blk[v * NB + bl];
          QR[v] = blk[v * NB + bl + stk];
        }
        rusanov<D>(QL, QR, k, p.gamma, G);
#pragma unroll
        for (int v = 0; v < NV; ++v) F[v * NFK + e] = G[v];
      }
      __syncthreads();
      const int kst = (k == 0) ? 1 : (k == 1 ? Ns : Ns * Ns);   // stride of axis k
      for (int e = tid; e < NV * NSD; e += nth) {
        const int v = e / NSD;
        int s = e - v * NSD, flo = 0, mul = 1;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          flo += (s % Ns) * mul;
          s /= Ns;
          mul *= (a == k) ? Ns + 1 : Ns;
        }
        A[e] -= ck * (F[v * NFK + flo + kst] - F[v * NFK + flo]);
      }
      // cell-face fluxes: edge[t][k][side][v][NSF]
      for (int e = tid; e < 2 * NV * NSF; e += nth) {
        const int side = e / (NV * NSF);
        const int r = e - side * NV * NSF;
        const int v = r / NSF, ts = r - v * NSF;
        const int tc[2] = {ts % Ns, ts / Ns};
        int fidx = 0, mul = 1, q = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const int cc = (a == k) ? (side ? Ns : 0) : tc[q++];
          fidx += cc * mul;
          mul *= (a == k) ? Ns + 1 : Ns;
        }
        p.b.edge[((size_t)t * D * 2 + (size_t)k * 2 + side) * NV * NSF + r] = F[v * NFK + fidx];
      }
    }
    __syncthreads();
    double* st = p.b.store[nxt] + (size_t)t * NV * NSD;
    for (int e = tid; e < NV * NSD; e += nth) st[e] = A[e];
    double lam = 0.0;
    const bool bad = check_subcells<D>(A, NSD, nullptr, p.gamma, mm, p.lam_mode ? &lam : nullptr, red,
                                       p.prec == ADG_PREC_MIXED_FP32, p.gam2f);
    if (tid == 0) {
      if (p.lam_mode) p.b.lam[cell] = lam;
      if (bad) atomicAdd(&p.b.counters[CNT_INADM], 1);
    }
    if (tid < 2 * NV) p.b.cmm[nxt][cell * 2 * NV + tid] = mm[tid];
    __syncthreads();
    double* u = apply_ct<D, NV, Ns, n>(A, B, R1, tid, nth);
    double* Uo = p.b.U[nxt] + cell * (NV * ND);
    for (int e = tid; e < NV * ND; e += nth) Uo[e] = u[e];
    if (tid == 0 && p.b.vok) p.b.vok[cell] = 0;     // P(R(v)) is not v: recompute next step
    if (tid < 2 * D) {
      const int k = tid >> 1, side = (tid & 1) ? 1 : -1;
      int nb[3];
      if (face_neighbour<D>(g, ijk, k, side, nb)) {
        const long long nc = cell_index<D>(nb, g);
        if (p.b.beta[nxt][nc]) {
          const int sl = p.b.slot[nxt][nc];
          // fixstamp marks unlimited cells for k_lim_fix; troubled cells are
          // never in that list, so it marks the WENO3 neighbours here
          if (sl >= 0 && p.b.fbflag[sl] != p.stamp) {
            const int old = atomicExch(&p.b.fixstamp[nc], p.stamp);
            if (old != p.stamp) {
              const int idx = atomicAdd(&p.b.counters[CNT_REFIX], 1);
              p.b.refixlist[idx] = (int)nc;
            }
          }
        }
      }
    }
  }
}

// Cascade layer, part 2: a WENO3 cell with fallback face neighbours takes
// their first-order flux on each shared face.  Its subcells next to such a
// face change by -+(dt/h_k)(F_first - F_weno), applied in the order axis 0
// low, axis 0 high, axis 1 low, ...; then min / max, wave speed and u = R(v)
// again.  One block per cell.
template <int D, int N>
__global__ void __launch_bounds__(128) k_lim_refix(Batch bt) {
  using DM = Dims<D, N>;
  constexpr int n = DM::n, NV = DM::NV, ND = DM::ND, Ns = DM::Ns, NSD = DM::NSD, NSF = DM::NSF;
  constexpr size_t EDGE = (size_t)D * 2 * NV * NSF;
  extern __shared__ double sm[];
  double* A = sm;                   // NV * NSD
  double* B = A + NV * NSD;         // NV * NSD
  double* R1 = B + NV * NSD;        // n * Ns
  double* mm = R1 + n * Ns;         // 2 NV
  double* red = mm + 2 * NV;        // 128
  __shared__ int fbslot[6];         // slot of the fallback neighbour per face, -1: none
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int i = tid; i < n * Ns; i += nth) R1[i] = bt.pps[0]->ops->R1[i];
  for (long long fg = blockIdx.x; fg < bt.pre[bt.n]; fg += gridDim.x) {
    const int sidx = batch_state(bt, fg);
    const Params& p = *bt.pps[sidx];
    const long long f = fg - bt.pre[sidx];
    const int nxt = 1 - p.cur;
    const Geo& g = p.geo;
    const long long cell = p.b.refixlist[f];
    const int t = p.b.slot[nxt][cell];
    int ijk[3];
    cell_coords<D>(cell, g, ijk);
    __syncthreads();
    if (tid < 2 * D) {
      const int k = tid >> 1, side = (tid & 1) ? 1 : -1;
      int nb[3], fs = -1;
      if (face_neighbour<D>(g, ijk, k, side, nb)) {
        const long long nc = cell_index<D>(nb, g);
        if (p.b.beta[nxt][nc]) {
          const int sl = p.b.slot[nxt][nc];
          if (sl >= 0 && p.b.fbflag[sl] == p.stamp) fs = sl;
        }
      }
      fbslot[tid] = fs;
    }
    double* st = p.b.store[nxt] + (size_t)t * NV * NSD;
    __syncthreads();
    const double* Et = p.b.edge + (size_t)t * EDGE;
    for (int e = tid; e < NV * NSD; e += nth) {
      const int v = e / NSD;
      int s = e - v * NSD;
      int sc[3] = {0, 0, 0};
#pragma unroll
      for (int a = 0; a < D; ++a) {
        sc[a] = s % Ns;
        s /= Ns;
      }
      double val = st[e];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const double ck = p.b.coef[3 + k];
        int ts = 0, mul = 1;
#pragma unroll
        for (int a = 0; a < D; ++a)
          if (a != k) {
            ts += sc[a] * mul;
            mul *= Ns;
          }
#pragma unroll
        for (int own = 0; own < 2; ++own) {
          const int fs = fbslot[2 * k + own];
          if (fs < 0 || sc[k] != (own ? Ns - 1 : 0)) continue;
          const double Fnew = p.b.edge[(size_t)fs * EDGE + ((size_t)k * 2 + (1 - own)) * NV * NSF + v * NSF + ts];
          const double Fold = Et[((size_t)k * 2 + own) * NV * NSF + v * NSF + ts];
          const double diff = ck * (Fnew - Fold);
          if (own) val -= diff;
          else val += diff;
        }
      }
      A[e] = val;
      st[e] = val;
    }
    __syncthreads();
    double lam = 0.0;
    const bool bad = check_subcells<D>(A, NSD, nullptr, p.gamma, mm, p.lam_mode ? &lam : nullptr, red,
                                       p.prec == ADG_PREC_MIXED_FP32, p.gam2f);
    if (tid == 0) {
      if (p.lam_mode) p.b.lam[cell] = lam;
      if (bad) atomicAdd(&p.b.counters[CNT_INADM], 1);
    }
    if (tid < 2 * NV) p.b.cmm[nxt][cell * 2 * NV + tid] = mm[tid];
    __syncthreads();
    double* u = apply_ct<D, NV, Ns, n>(A, B, R1, tid, nth);
    double* Uo = p.b.U[nxt] + cell * (NV * ND);
    for (int e = tid; e < NV * ND; e += nth) Uo[e] = u[e];
    if (tid == 0 && p.b.vok) p.b.vok[cell] = 0;     // P(R(v)) is not v: recompute next step
  }
}

}  // namespace adg
