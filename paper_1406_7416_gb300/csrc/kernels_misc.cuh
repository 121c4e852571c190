// Load-time kernels (initial detection, full-state load / read), the device
// projection of the test problems' initial data, and the time-step reduction.
#pragma once

#include "kernels_lim.cuh"

namespace adg {

// Initial detection (Sec. 4.4, last paragraph) or plain load.  One cell per
// block.  `exact` (device [cells][nv][Ns^d]) may be null: no detection.
// cmm_ex: per-cell min/max of the exact averages (used when exact != null).
template <int D, int N>
__global__ void __launch_bounds__(128) k_load_detect(Params p, const double* __restrict__ exact,
                                                     const double* __restrict__ cmm_ex) {
  using DM = Dims<D, N>;
  constexpr int n = DM::n, NV = DM::NV, ND = DM::ND, Ns = DM::Ns, NSD = DM::NSD;
  extern __shared__ double sm[];
  double* A = sm;
  double* B = A + NV * NSD;
  double* P1 = B + NV * NSD;
  double* R1 = P1 + Ns * n;
  double* lohi = R1 + n * Ns;
  double* mm = lohi + 2 * NV;
  double* red = mm + 2 * NV;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int i = tid; i < Ns * n; i += nth) {
    P1[i] = p.ops->P1[i];
    R1[i] = p.ops->R1[i];
  }
  __shared__ int s_slot;
  const int cur = p.cur;
  for (long long cell = blockIdx.x; cell < p.geo.cells; cell += gridDim.x) {
    int ijk[3];
    cell_coords<D>(cell, p.geo, ijk);
    double* U = p.b.U[cur] + cell * (NV * ND);
    __syncthreads();
    for (int e = tid; e < NV * ND; e += nth) A[e] = U[e];
    __syncthreads();
    double* vs = apply_ct<D, NV, n, Ns>(A, B, P1, tid, nth);
    if (exact) dmp_interval<D>(p, cmm_ex, ijk, lohi);
    __syncthreads();
    double lam;
    const bool troubled = check_subcells<D>(vs, NSD, exact ? lohi : nullptr, p.gamma, mm, &lam, red)
                          && exact != nullptr;
    if (!troubled) {
      if (tid == 0) {
        p.b.beta[cur][cell] = 0;
        p.b.slot[cur][cell] = -1;
        p.b.lam[cell] = lam;
      }
      if (tid < 2 * NV) p.b.cmm[cur][cell * 2 * NV + tid] = mm[tid];
      continue;
    }
    // flagged at t = 0: keep the exact averages, DOFs become R(exact)
    if (tid == 0) {
      int slot = atomicAdd(&p.b.counters[CNT_TROUBLED0 + cur], 1);
      if (slot < p.cap) {
        p.b.list[cur][slot] = (int)cell;
      } else {
        atomicOr(&p.b.counters[CNT_STATUS], 1);
        slot = -1;
      }
      s_slot = slot;
    }
    __syncthreads();
    const int slot = s_slot;
    const double* ex = exact + cell * (size_t)(NV * NSD);
    if (slot < 0) {
      if (tid == 0) p.b.beta[cur][cell] = 0;
      continue;
    }
    double* st = p.b.store[cur] + (size_t)slot * NV * NSD;
    __syncthreads();
    for (int e = tid; e < NV * NSD; e += nth) {
      st[e] = ex[e];
      A[e] = ex[e];
    }
    __syncthreads();
    check_subcells<D>(A, NSD, nullptr, p.gamma, mm, &lam, red);
    double* u = apply_ct<D, NV, Ns, n>(A, B, R1, tid, nth);
    for (int e = tid; e < NV * ND; e += nth) U[e] = u[e];
    if (tid == 0) {
      p.b.beta[cur][cell] = 1;
      p.b.slot[cur][cell] = slot;
      p.b.lam[cell] = lam;
    }
    if (tid < 2 * NV) p.b.cmm[cur][cell * 2 * NV + tid] = mm[tid];
  }
}

// Wave speeds of the current level from v^n (stored subcell data of troubled
// cells, P(u^n) elsewhere), for a time step requested after steps that did
// not keep them current.
template <int D, int N>
__global__ void __launch_bounds__(128) k_lambda(Params p) {
  using DM = Dims<D, N>;
  constexpr int n = DM::n, NV = DM::NV, ND = DM::ND, Ns = DM::Ns, NSD = DM::NSD;
  extern __shared__ double sm[];
  double* A = sm;
  double* B = A + NV * NSD;
  double* P1 = B + NV * NSD;
  double* mm = P1 + Ns * n;
  double* red = mm + 2 * NV;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int i = tid; i < Ns * n; i += nth) P1[i] = p.ops->P1[i];
  const int cur = p.cur;
  for (long long cell = blockIdx.x; cell < p.geo.cells; cell += gridDim.x) {
    __syncthreads();
    double* vs;
    if (p.b.beta[cur][cell]) {
      const double* st = p.b.store[cur] + (size_t)p.b.slot[cur][cell] * NV * NSD;
      for (int e = tid; e < NV * NSD; e += nth) A[e] = st[e];
      __syncthreads();
      vs = A;
    } else {
      const double* U = p.b.U[cur] + cell * (NV * ND);
      for (int e = tid; e < NV * ND; e += nth) A[e] = U[e];
      __syncthreads();
      vs = apply_ct<D, NV, n, Ns>(A, B, P1, tid, nth);
    }
    double lam;
    check_subcells<D>(vs, NSD, nullptr, p.gamma, mm, &lam, red);
    if (tid == 0) p.b.lam[cell] = lam;
  }
}

// Per-cell min / max of subcell data sub[cells][nv][Ns^d] -> out[cells][nv][2]
template <int D, int N>
__global__ void k_sub_minmax(const double* __restrict__ sub, double* __restrict__ out,
                             long long cells) {
  using DM = Dims<D, N>;
  constexpr int NV = DM::NV, NSD = DM::NSD;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < cells * NV;
       e += (long long)gridDim.x * blockDim.x) {
    const double* s = sub + e * NSD;
    double mn = s[0], mx = s[0];
    for (int i = 1; i < NSD; ++i) {
      mn = fmin(mn, s[i]);
      mx = fmax(mx, s[i]);
    }
    out[2 * e] = mn;
    out[2 * e + 1] = mx;
  }
}

// Full-state load: flags given; flagged cells take their subcell rows.
template <int D, int N>
__global__ void __launch_bounds__(128) k_load_full(Params p, const uint8_t* __restrict__ beta,
                                                   const double* __restrict__ sub) {
  using DM = Dims<D, N>;
  constexpr int n = DM::n, NV = DM::NV, ND = DM::ND, Ns = DM::Ns, NSD = DM::NSD;
  extern __shared__ double sm[];
  double* A = sm;
  double* B = A + NV * NSD;
  double* P1 = B + NV * NSD;
  double* mm = P1 + Ns * n;
  double* red = mm + 2 * NV;
  __shared__ int s_slot;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int i = tid; i < Ns * n; i += nth) P1[i] = p.ops->P1[i];
  const int cur = p.cur;
  for (long long cell = blockIdx.x; cell < p.geo.cells; cell += gridDim.x) {
    __syncthreads();
    const bool flagged = beta[cell] != 0;
    double* vs;
    if (flagged) {
      if (tid == 0) {
        int slot = atomicAdd(&p.b.counters[CNT_TROUBLED0 + cur], 1);
        if (slot < p.cap) {
          p.b.list[cur][slot] = (int)cell;
        } else {
          atomicOr(&p.b.counters[CNT_STATUS], 1);
          slot = -1;
        }
        s_slot = slot;
      }
      __syncthreads();
      const int slot = s_slot;
      const double* src = sub + cell * (size_t)(NV * NSD);
      for (int e = tid; e < NV * NSD; e += nth) {
        A[e] = src[e];
        if (slot >= 0) p.b.store[cur][(size_t)slot * NV * NSD + e] = src[e];
      }
      if (tid == 0) {
        p.b.beta[cur][cell] = slot >= 0 ? 1 : 0;
        p.b.slot[cur][cell] = slot;
      }
      __syncthreads();
      vs = A;
    } else {
      const double* U = p.b.U[cur] + cell * (NV * ND);
      for (int e = tid; e < NV * ND; e += nth) A[e] = U[e];
      if (tid == 0) {
        p.b.beta[cur][cell] = 0;
        p.b.slot[cur][cell] = -1;
      }
      __syncthreads();
      vs = apply_ct<D, NV, n, Ns>(A, B, P1, tid, nth);
    }
    double lam;
    check_subcells<D>(vs, NSD, nullptr, p.gamma, mm, &lam, red);
    if (tid == 0) p.b.lam[cell] = lam;
    if (tid < 2 * NV) p.b.cmm[cur][cell * 2 * NV + tid] = mm[tid];
  }
}

// Subcell data of flagged cells -> sub[cells][nv][Ns^d] (NaN rows elsewhere)
template <int D, int N>
__global__ void k_read_full(Params p, double* __restrict__ sub) {
  using DM = Dims<D, N>;
  constexpr int NV = DM::NV, NSD = DM::NSD;
  const long long total = p.geo.cells * NV * NSD;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long cell = e / (NV * NSD);
    const int r = (int)(e - cell * (NV * NSD));
    double v = __longlong_as_double(0x7ff8000000000000LL);
    if (p.b.beta[p.cur][cell]) {
      const int slot = p.b.slot[p.cur][cell];
      if (slot >= 0) v = p.b.store[p.cur][(size_t)slot * NV * NSD + r];
    }
    sub[e] = v;
  }
}

// Primitive initial state at one point of a test problem (Sec. 5.2, 5.6, 5.8).
template <int D>
__device__ __forceinline__ void problem_state(const adg_problem& pr, const double* x, double fac,
                                              double gamma, double* Q) {
  double rho, vel[3] = {0.0, 0.0, 0.0}, p;
  if (pr.kind == ADG_IC_PLANAR) {
    double sdot = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) sdot += pr.normal[k] * x[k];
    const double* s = (sdot < pr.offset) ? pr.inner : pr.outer;
    rho = s[0] * fac;
#pragma unroll
    for (int k = 0; k < D; ++k) vel[k] = s[1 + k];
    p = s[1 + D];
  } else if (pr.kind == ADG_IC_RADIAL) {
    double r2 = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) r2 += (x[k] - pr.center[k]) * (x[k] - pr.center[k]);
    const double* s = (r2 <= pr.radius * pr.radius) ? pr.inner : pr.outer;
    rho = s[0] * fac;
#pragma unroll
    for (int k = 0; k < D; ++k) vel[k] = s[1 + k];
    p = s[1 + D];
  } else {
    const bool right = x[0] > pr.center[0], up = x[1] > pr.center[1];
    const int q = right ? (up ? 0 : 3) : (up ? 1 : 2);
    rho = pr.quad[q][0];
    vel[0] = pr.quad[q][1];
    vel[1] = pr.quad[q][2];
    p = pr.quad[q][3];
    if (pr.vortex) {
      const double xp = x[0] - pr.vortex_center[0], yp = x[1] - pr.vortex_center[1];
      const double r2 = xp * xp + yp * yp;
      const double b = pr.vortex_strength;
      const double e = exp(0.5 * (1.0 - r2));
      const double pi = 3.14159265358979323846;
      // temperature perturbation with beta^2 (radial equilibrium of the vortex)
      const double dT = -(gamma - 1.0) * b * b / (8.0 * gamma * pi * pi) * e * e;
      const double T0 = p / rho;
      const double T = T0 + dT;
      rho = rho * pow(T / T0, 1.0 / (gamma - 1.0));
      p = rho * T;
      vel[0] += -yp * b / (2.0 * pi) * e;
      vel[1] += xp * b / (2.0 * pi) * e;
    }
  }
  Q[0] = rho;
  double kin = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    Q[1 + k] = rho * vel[k];
    kin += vel[k] * vel[k];
  }
  Q[1 + D] = p / (gamma - 1.0) + 0.5 * rho * kin;
}

// L2 projection of the initial data (composite rule: Ns subintervals x
// (N+2) GL points per axis) and exact subcell averages.  One cell per block;
// rows of points along x are reduced first, then accumulated.
template <int D, int N>
__global__ void __launch_bounds__(128) k_project(Params p, adg_problem pr,
                                                 const double* __restrict__ fac,
                                                 double* __restrict__ exact) {
  using DM = Dims<D, N>;
  constexpr int n = DM::n, NV = DM::NV, ND = DM::ND, Ns = DM::Ns, NSD = DM::NSD;
  constexpr int Q1 = N + 2, NQ = Ns * Q1;
  __shared__ double row[NV][NQ];
  __shared__ double tx[NV][n];
  __shared__ double sx[NV][Ns];
  __shared__ double Ua[NV * ND];
  __shared__ double Va[NV * NSD];
  const Ops* o = p.ops;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int nrows = (D == 3) ? NQ * NQ : NQ;
  for (long long cell = blockIdx.x; cell < p.geo.cells; cell += gridDim.x) {
    int ijk[3];
    cell_coords<D>(cell, p.geo, ijk);
    const double f = fac ? fac[cell] : 1.0;
    __syncthreads();
    if (pr.kind == ADG_IC_RADIAL) {
      // a cell wholly inside or outside the sphere holds one constant state,
      // whose projection and subcell averages are that state (what the
      // composite rule gives up to rounding); only cut cells need the rule
      double rmin2 = 0.0, rmax2 = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const double lo = p.geo.x0[k] + ijk[k] * p.geo.dx[k] - pr.center[k];
        const double hi = lo + p.geo.dx[k];
        const double near = (lo > 0.0) ? lo : (hi < 0.0 ? -hi : 0.0);
        const double far = fmax(fabs(lo), fabs(hi));
        rmin2 += near * near;
        rmax2 += far * far;
      }
      const double R2 = pr.radius * pr.radius;
      if (rmax2 < R2 * (1.0 - 1e-12) || rmin2 > R2 * (1.0 + 1e-12)) {
        double x[3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
          x[k] = (k < D) ? p.geo.x0[k] + (ijk[k] + 0.5) * p.geo.dx[k] : 0.0;
        double Q[NV];
        problem_state<D>(pr, x, f, p.gamma, Q);
        double* U = p.b.U[p.cur] + cell * (NV * ND);
        for (int e = tid; e < NV * ND; e += nth) U[e] = Q[e / ND];
        double* ex = exact + cell * (size_t)(NV * NSD);
        for (int e = tid; e < NV * NSD; e += nth) ex[e] = Q[e / NSD];
        continue;
      }
    }
    for (int e = tid; e < NV * ND; e += nth) Ua[e] = 0.0;
    for (int e = tid; e < NV * NSD; e += nth) Va[e] = 0.0;
    for (int rw = 0; rw < nrows; ++rw) {
      const int qy = rw % NQ, qz = rw / NQ;
      __syncthreads();
      for (int px = tid; px < NQ; px += nth) {
        double x[3];
        x[0] = p.geo.x0[0] + (ijk[0] + o->cq_x[px]) * p.geo.dx[0];
        x[1] = p.geo.x0[1] + (ijk[1] + o->cq_x[qy]) * p.geo.dx[1];
        x[2] = (D == 3) ? p.geo.x0[2] + (ijk[2] + o->cq_x[qz]) * p.geo.dx[2] : 0.0;
        double Q[NV];
        problem_state<D>(pr, x, f, p.gamma, Q);
#pragma unroll
        for (int v = 0; v < NV; ++v) row[v][px] = Q[v];
      }
      __syncthreads();
      // reduce the row along x: DOF weights and subcell averages
      for (int e = tid; e < NV * (n + Ns); e += nth) {
        const int v = e / (n + Ns), r = e - v * (n + Ns);
        double acc = 0.0;
        if (r < n) {
          for (int q = 0; q < NQ; ++q) acc += o->cq_w[q] * o->cq_phi[q * n + r] * row[v][q];
          tx[v][r] = acc / o->w[r];
        } else {
          const int s = r - n;
          for (int q = s * Q1; q < (s + 1) * Q1; ++q) acc += o->cq_w[q] * Ns * row[v][q];
          sx[v][s] = acc;
        }
      }
      __syncthreads();
      const double wy = o->cq_w[qy], wz = (D == 3) ? o->cq_w[qz] : 1.0;
      for (int e = tid; e < NV * ND; e += nth) {
        const int v = e / ND;
        int i = e - v * ND;
        const int a = i % n, b = (i / n) % n, c = (D == 3) ? i / (n * n) : 0;
        double wgt = wy * o->cq_phi[qy * n + b] / o->w[b];
        if (D == 3) wgt *= wz * o->cq_phi[qz * n + c] / o->w[c];
        Ua[e] += wgt * tx[v][a];
      }
      const int sy = qy / Q1, sz = (D == 3) ? qz / Q1 : 0;
      for (int e = tid; e < NV * Ns; e += nth) {
        const int v = e / Ns, s = e - v * Ns;
        double wgt = wy * Ns;
        if (D == 3) wgt *= wz * Ns;
        Va[v * NSD + s + Ns * (sy + Ns * sz)] += wgt * sx[v][s];
      }
    }
    __syncthreads();
    double* U = p.b.U[p.cur] + cell * (NV * ND);
    for (int e = tid; e < NV * ND; e += nth) U[e] = Ua[e];
    double* ex = exact + cell * (size_t)(NV * NSD);
    for (int e = tid; e < NV * NSD; e += nth) ex[e] = Va[e];
  }
}

}  // namespace adg

namespace adg {

// ---------------------------------------------------------------------------
// Halo exchange of a domain decomposition (the paper's MPI runs split the
// grid among processes and exchange neighbour data every step, Sec. 5.8;
// the flux correction of Sec. 4.4 couples cells across a partition edge).
// A box of cells [lo, hi) of one state is packed into a caller buffer with
// the level-n data another state needs to step cells beyond its own: DOFs,
// flags, the stored subcell data of flagged cells and the per-cell extrema
// of the subcell data (the DMP bounds' inputs).  Packed layout, for count
// cells in box order (x fastest):
//   dofs [count][nv][n^d] | sub [count][nv][Ns^d] | cmm [count][nv][2] |
//   beta [count] bytes
// ---------------------------------------------------------------------------
struct Box {
  int lo[3], hi[3];
  long long count;
};

template <int D>
__device__ __forceinline__ long long box_cell(const Box& bx, long long q, const Geo& g) {
  const int ex = bx.hi[0] - bx.lo[0], ey = bx.hi[1] - bx.lo[1];
  int ijk[3];
  ijk[0] = bx.lo[0] + (int)(q % ex);
  const long long r = q / ex;
  ijk[1] = bx.lo[1] + (int)(r % ey);
  ijk[2] = D == 3 ? bx.lo[2] + (int)(r / ey) : 0;
  return cell_index<D>(ijk, g);
}

// position of local cell c in the box, or -1
template <int D>
__device__ __forceinline__ long long box_index(const Box& bx, long long c, const Geo& g) {
  int ijk[3];
  cell_coords<D>(c, g, ijk);
  long long q = 0, mul = 1;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    if (ijk[k] < bx.lo[k] || ijk[k] >= bx.hi[k]) return -1;
    q += (ijk[k] - bx.lo[k]) * mul;
    mul *= bx.hi[k] - bx.lo[k];
  }
  return q;
}

template <int D, int N>
struct Packed {
  using DM = Dims<D, N>;
  static constexpr int NV = DM::NV, ND = DM::ND, NSD = DM::NSD;
  double* dofs;
  double* sub;
  double* cmm;
  uint8_t* beta;
  __host__ __device__ Packed(void* buf, long long count) {
    dofs = static_cast<double*>(buf);
    sub = dofs + count * NV * ND;
    cmm = sub + count * NV * NSD;
    beta = reinterpret_cast<uint8_t*>(cmm + count * 2 * NV);
  }
  static size_t bytes(long long count) {
    return (size_t)count * ((NV * ND + NV * NSD + 2 * NV) * sizeof(double) + 1);
  }
};

// One block per box cell: the level-n data of the cell into the buffer.
template <int D, int N>
__global__ void __launch_bounds__(128) k_pack(Params p, Box bx, void* buf) {
  using PK = Packed<D, N>;
  constexpr int NV = PK::NV, ND = PK::ND, NSD = PK::NSD;
  PK pk(buf, bx.count);
  const int cur = p.cur;
  for (long long q = blockIdx.x; q < bx.count; q += gridDim.x) {
    const long long c = box_cell<D>(bx, q, p.geo);
    const double* U = p.b.U[cur] + c * (NV * ND);
    for (int e = threadIdx.x; e < NV * ND; e += blockDim.x) pk.dofs[q * NV * ND + e] = U[e];
    for (int e = threadIdx.x; e < 2 * NV; e += blockDim.x)
      pk.cmm[q * 2 * NV + e] = p.b.cmm[cur][c * 2 * NV + e];
    const uint8_t b = p.b.beta[cur][c];
    const int slot = p.b.slot[cur][c];
    if (threadIdx.x == 0) pk.beta[q] = (b && slot >= 0) ? 1 : 0;
    if (b && slot >= 0) {
      const double* src = p.b.store[cur] + (size_t)slot * NV * NSD;
      for (int e = threadIdx.x; e < NV * NSD; e += blockDim.x) pk.sub[q * NV * NSD + e] = src[e];
    }
  }
}

// One block per box cell: DOFs, flags and extrema of the buffer become the
// cell's level n; its kept subcell averages (mixed precision) are dropped.
template <int D, int N>
__global__ void __launch_bounds__(128) k_unpack(Params p, Box bx, const void* buf) {
  using PK = Packed<D, N>;
  constexpr int NV = PK::NV, ND = PK::ND;
  const PK pk(const_cast<void*>(buf), bx.count);
  const int cur = p.cur;
  for (long long q = blockIdx.x; q < bx.count; q += gridDim.x) {
    const long long c = box_cell<D>(bx, q, p.geo);
    double* U = p.b.U[cur] + c * (NV * ND);
    for (int e = threadIdx.x; e < NV * ND; e += blockDim.x) U[e] = pk.dofs[q * NV * ND + e];
    for (int e = threadIdx.x; e < 2 * NV; e += blockDim.x)
      p.b.cmm[cur][c * 2 * NV + e] = pk.cmm[q * 2 * NV + e];
    if (threadIdx.x == 0) {
      p.b.beta[cur][c] = pk.beta[q];
      if (p.b.vok) p.b.vok[c] = 0;
    }
  }
}

// One block per cell: the level-n troubled list rebuilt into the other
// level's (dead) list, slot and store arrays, rows of box cells taken from
// the buffer and the others from their current slots; the counter of the
// other level (zeroed by the host, reset again by the next step begin) counts.
template <int D, int N>
__global__ void __launch_bounds__(128) k_relist(Params p, Box bx, const void* buf) {
  using PK = Packed<D, N>;
  constexpr int NV = PK::NV, NSD = PK::NSD;
  const PK pk(const_cast<void*>(buf), bx.count);
  const int cur = p.cur, nxt = 1 - cur;
  __shared__ int s_slot;
  for (long long c = blockIdx.x; c < p.geo.cells; c += gridDim.x) {
    const uint8_t b = p.b.beta[cur][c];
    if (!b) {
      if (threadIdx.x == 0) p.b.slot[nxt][c] = -1;
      continue;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int s = atomicAdd(&p.b.counters[CNT_TROUBLED0 + nxt], 1);
      if (s < p.cap) {
        p.b.list[nxt][s] = (int)c;
      } else {
        atomicOr(&p.b.counters[CNT_STATUS], 1);
        s = -1;
      }
      p.b.slot[nxt][c] = s;
      s_slot = s;
    }
    __syncthreads();
    const int s = s_slot;
    if (s < 0) continue;
    const long long q = box_index<D>(bx, c, p.geo);
    const double* src = q >= 0 ? pk.sub + q * NV * NSD
                               : p.b.store[cur] + (size_t)p.b.slot[cur][c] * NV * NSD;
    double* dst = p.b.store[nxt] + (size_t)s * NV * NSD;
    for (int e = threadIdx.x; e < NV * NSD; e += blockDim.x) dst[e] = src[e];
  }
}

// The rebuilt list, slots and stored rows copied back to level n.
template <int D, int N>
__global__ void k_copyback(Params p) {
  constexpr int NV = D + 2, NSD = ipow(2 * N + 1, D);
  const int cur = p.cur, nxt = 1 - cur;
  int n = p.b.counters[CNT_TROUBLED0 + nxt];
  if (n > p.cap) n = p.cap;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = t0; e < (long long)n * NV * NSD; e += stride)
    p.b.store[cur][e] = p.b.store[nxt][e];
  for (long long e = t0; e < n; e += stride) p.b.list[cur][e] = p.b.list[nxt][e];
  for (long long c = t0; c < p.geo.cells; c += stride) {
    p.b.slot[cur][c] = p.b.slot[nxt][c];
    if (p.b.slot[cur][c] < 0) p.b.beta[cur][c] = 0;      // no slot left: the cell is unflagged
  }
  if (t0 == 0) p.b.counters[CNT_TROUBLED0 + cur] = n;
}

}  // namespace adg
