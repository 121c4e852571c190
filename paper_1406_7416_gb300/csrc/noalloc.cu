// Subcell ADER-WENO3 update of caller-owned patches with no device allocation.
//
// All scratch of this entry point (WENO sweeps, subcell space-time
// predictors, sub-face fluxes, the operator table, a few control words) lives
// in one file-scope static device array of NOALLOC_SCRATCH_BYTES.  Every GPU
// that loads libadg holds that array until the process exits.  Host code
// cannot use the array's name as a device address: the address is looked up
// once per device with cudaGetSymbolAddress, with that device current, on the
// first call made while it is current.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "launch.cuh"

namespace adg {
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;    // 32 MiB
// Control block, each region in its own 128-byte slot:
//   [0, 64)     counters (CNT_COUNT ints)
//   [64, 192)   dt[0], lamred dt[1], clock dt[2..4], dt / dx_k at dt[6..8],
//               dt Ns / dx_k at dt[9..11] (12 doubles)
//   [192, 256)  the one-state pointer array of the batch descriptor
//   [256, 320)  the item prefix pre[0..1]
// then the Params, the operator table and the buffers.
constexpr size_t CTRL_COUNTERS = 0, CTRL_DT = 64, CTRL_PPS = 192, CTRL_PRE = 256;
constexpr size_t CTRL_BYTES = 512;
constexpr int CTRL_DT_WORDS = 12;
static_assert(CNT_COUNT * sizeof(int) <= CTRL_DT - CTRL_COUNTERS, "counters overlap dt");
static_assert(CTRL_DT + CTRL_DT_WORDS * sizeof(double) <= CTRL_PPS, "dt words overlap pps");
static_assert(CTRL_PPS + sizeof(Params*) <= CTRL_PRE, "pps overlaps pre");
static_assert(CTRL_PRE + 2 * sizeof(long long) <= CTRL_BYTES, "pre overlaps the Params");
constexpr size_t PARAMS_BYTES = (sizeof(Params) + 255) / 256 * 256;
constexpr size_t OPS_BYTES = (sizeof(Ops) + 255) / 256 * 256 + PARAMS_BYTES;
constexpr int MAX_DEVICES = 64;

// The Params and the operator table of one call, laid out as in the static
// area (Params at CTRL_BYTES, Ops PARAMS_BYTES after it), so that one copy
// uploads both.
struct alignas(256) Upload {
  unsigned char bytes[PARAMS_BYTES + sizeof(Ops)];
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_setup_mutex;
unsigned char* g_device_base[MAX_DEVICES] = {};

// Start-of-call control words: counters cleared, troubled count and dt set,
// a one-state batch descriptor whose items are the `count` patches.
__global__ void k_noalloc_begin(int* counters, double* dt, Params** pps, long long* pre,
                                Params* params, int count, double dtv) {
  if (threadIdx.x < CNT_COUNT) counters[threadIdx.x] = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    counters[CNT_TROUBLED1] = count;
    dt[0] = dtv;
    dt[1] = 0.0;
    dt[2] = 0.0;
    dt[3] = 0.0;
    // dt / dx_k and dt Ns / dx_k as the step kernels read them (dt + 6)
    const int Ns = 2 * params->N + 1;
    for (int k = 0; k < params->dim; ++k) {
      dt[6 + k] = dtv / params->geo.dx[k];
      dt[9 + k] = dtv * Ns / params->geo.dx[k];
    }
    pps[0] = params;
    pre[0] = 0;
    pre[1] = count;
  }
}

// Finite volume update of the interior subcells and the sub-face fluxes on the
// cell faces, written to the caller's buffers.
template <int D, int N>
__global__ void k_noalloc_write(Params p, int count, double* __restrict__ vnew,
                                double* __restrict__ faces) {
  using DM = Dims<D, N>;
  constexpr int NV = DM::NV, Ns = DM::Ns, NSD = DM::NSD, L = DM::L, LD = DM::LD, NSF = DM::NSF;
  constexpr int NFK = (Ns + 1) * NSF;
  const double dt = *p.b.dt;
  double c[3];
#pragma unroll
  for (int k = 0; k < D; ++k) c[k] = dt * Ns / p.geo.dx[k];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)count * NV * NSD;
       e += (long long)gridDim.x * blockDim.x) {
    const long long jv = e / NSD;
    const long long j = jv / NV;
    const int v = (int)(jv - j * NV);
    int s = (int)(e - jv * NSD);
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
    double val = p.b.patch[(j * NV + v) * LD + poff];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      int flo = 0, mul = 1;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        flo += sc[a] * mul;
        mul *= (a == k) ? Ns + 1 : Ns;
      }
      const int kst = (k == 0) ? 1 : (k == 1 ? Ns : Ns * Ns);
      const double* F = p.b.fsub[k] + (j * NV + v) * NFK;
      val -= c[k] * (F[flo + kst] - F[flo]);
    }
    vnew[e] = val;
  }
  if (!faces) return;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
       e < (long long)count * D * 2 * NV * NSF; e += (long long)gridDim.x * blockDim.x) {
    const long long j = e / (D * 2 * NV * NSF);
    int r = (int)(e - j * (D * 2 * NV * NSF));
    const int k = r / (2 * NV * NSF);
    r -= k * 2 * NV * NSF;
    const int side = r / (NV * NSF);
    r -= side * NV * NSF;
    const int v = r / NSF, ts = r - v * NSF;
    const int tc[2] = {ts % Ns, ts / Ns};
    int fidx = 0, mul = 1, q = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int cc = (a == k) ? (side ? Ns : 0) : tc[q++];
      fidx += cc * mul;
      mul *= (a == k) ? Ns + 1 : Ns;
    }
    faces[e] = p.b.fsub[k][(j * NV + v) * NFK + fidx];
  }
}

template <int D, int N>
struct NoAlloc {
  using DM = Dims<D, N>;

  static size_t per_cell_bytes() {
    size_t a, b, c, d, e, f;
    scratch_of<D, N>(&a, &b, &c, &d, &e, &f);
    return (b + c + d + e + D * f) * sizeof(double);
  }

  static cudaError_t run(Params p, Params* pdev, Params** pps, long long* pre, int count,
                         double dt, double* vnew, double* faces, cudaStream_t s) {
    k_noalloc_begin<<<1, 32, 0, s>>>(p.b.counters, p.b.dt, pps, pre, pdev, count, dt);
    if (count == 0) return cudaGetLastError();
    constexpr int SPB = (D == 2) ? SUBS_PER_BLOCK_2D : SUBS_PER_BLOCK_3D;
    const long long ch = count;
    const Batch lim{pps, 1, pre};
    k_lim_sweep<D, N, 0, double><<<grid_for(ch * DM::NV * DM::LD, 256), 256, 0, s>>>(lim, 0);
    k_lim_sweep<D, N, 1, double><<<grid_for(ch * DM::NV * DM::LD, 256), 256, 0, s>>>(lim, 0);
    if (D == 3)
      k_lim_sweep<D, N, (D == 3 ? 2 : 1), double><<<grid_for(ch * DM::NV * DM::LD, 256), 256, 0, s>>>(lim, 0);
    const long long ncross = ch * (DM::NSD + 2 * D * DM::NSF);
    k_lim_predict<D, N, false, double, false><<<grid_for(ncross, SPB, kNumSM * 16), SPB * DM::NST3, 0, s>>>(lim, 0, 0);
    k_lim_flux<D, N, 0, double, double><<<grid_for(ch * (DM::Ns + 1) * DM::NSF, 256), 256, 0, s>>>(lim, 0);
    k_lim_flux<D, N, 1, double, double><<<grid_for(ch * (DM::Ns + 1) * DM::NSF, 256), 256, 0, s>>>(lim, 0);
    if (D == 3)
      k_lim_flux<D, N, (D == 3 ? 2 : 1), double, double><<<grid_for(ch * (DM::Ns + 1) * DM::NSF, 256), 256, 0, s>>>(
          lim, 0);
    k_noalloc_write<D, N><<<grid_for(ch * DM::NV * DM::NSD, 256), 256, 0, s>>>(p, count, vnew, faces);
    return cudaGetLastError();
  }

  // Carve the static scratch into the limiter's chunk buffers for `count` cells.
  static void carve(unsigned char* base, int count, Params& p) {
    size_t a, b, c, d, e, f;
    scratch_of<D, N>(&a, &b, &c, &d, &e, &f);
    double* q = reinterpret_cast<double*>(base + CTRL_BYTES + OPS_BYTES);
    p.b.sweep[0] = q;
    q += (size_t)count * b;
    p.b.sweep[1] = q;
    q += (size_t)count * c;
    p.b.sweep[2] = (D == 3) ? q : nullptr;
    q += (size_t)count * d;
    p.b.qsub = q;
    q += (size_t)count * e;
    for (int k = 0; k < D; ++k) {
      p.b.fsub[k] = q;
      q += (size_t)count * f;
    }
  }
};

template <int D, int N>
int run_noalloc(unsigned char* base, double gamma, const double* h, double dt, const double* patches,
                int count, double* vnew, double* faces, cudaStream_t s, char* err, size_t errlen) {
  using NA = NoAlloc<D, N>;
  const size_t need = CTRL_BYTES + OPS_BYTES + (size_t)count * NA::per_cell_bytes();
  if (need > NOALLOC_SCRATCH_BYTES) {
    if (err && errlen)
      snprintf(err, errlen,
               "adg_subcell_update_noalloc: %d patches need %zu bytes of scratch, the static "
               "area holds %zu (at most %zu patches for dim=%d, N=%d)",
               count, need, NOALLOC_SCRATCH_BYTES,
               (NOALLOC_SCRATCH_BYTES - CTRL_BYTES - OPS_BYTES) / NA::per_cell_bytes(), D, N);
    return ADG_ERR_CAPACITY;
  }
  Upload up;
  Ops& ops_host = *reinterpret_cast<Ops*>(up.bytes + PARAMS_BYTES);
  build_ops(N, &ops_host);
  Params* params_dev = reinterpret_cast<Params*>(base + CTRL_BYTES);
  Ops* ops_dev = reinterpret_cast<Ops*>(base + CTRL_BYTES + PARAMS_BYTES);
  Params p;
  memset(&p, 0, sizeof(Params));
  p.geo.dim = D;
  for (int k = 0; k < 3; ++k) {
    p.geo.n[k] = 1;
    p.geo.dx[k] = (k < D) ? h[k] * (2 * N + 1) : 1.0;   // kernels use dt * Ns / dx = dt / h
  }
  p.N = N;
  p.dim = D;
  p.nv = D + 2;
  p.prec = ADG_PREC_FP64;
  p.iters = N + 1;
  p.fp64_sweeps = 1;
  p.cap = count;
  p.chunk = count > 0 ? count : 1;
  p.gamma = gamma;
  p.ops = ops_dev;
  p.cur = 0;
  p.b.counters = reinterpret_cast<int*>(base + CTRL_COUNTERS);
  p.b.dt = reinterpret_cast<double*>(base + CTRL_DT);
  p.b.lamred = p.b.dt + 1;
  p.b.clock = p.b.dt + 2;
  p.b.coef = p.b.dt + 6;
  p.b.patch = const_cast<double*>(patches);
  NA::carve(base, count, p);
  memcpy(up.bytes, &p, sizeof(Params));
  // one upload of the Params and the operator table, then one wait: `up`
  // lives on this stack frame
  cudaError_t e = cudaMemcpyAsync(params_dev, up.bytes, sizeof(up.bytes), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    if (err && errlen) snprintf(err, errlen, "parameter upload failed: %s", cudaGetErrorString(e));
    return ADG_ERR_CUDA;
  }
  e = NA::run(p, params_dev, reinterpret_cast<Params**>(base + CTRL_PPS),
              reinterpret_cast<long long*>(base + CTRL_PRE), count, dt, vnew, faces, s);
  if (e != cudaSuccess) {
    if (err && errlen) snprintf(err, errlen, "kernel launch failed: %s", cudaGetErrorString(e));
    return ADG_ERR_CUDA;
  }
  return ADG_OK;
}

}  // namespace
}  // namespace adg

using namespace adg;

extern "C" int adg_subcell_update_noalloc(int dim, int N, double gamma, const double* h, double dt,
                                          const double* patches, int count, double* vnew,
                                          double* faces, void* stream, char* err, size_t errlen) {
  if (err && errlen) err[0] = '\0';
  auto bad = [&](const char* msg) {
    if (err && errlen) snprintf(err, errlen, "adg_subcell_update_noalloc: %s", msg);
    return ADG_ERR_ARG;
  };
  if (dim != 2 && dim != 3) return bad("dim must be 2 or 3");
  if (N < 1 || N > 9 || (dim == 3 && N > 3)) return bad("N must be 1..9 (2D) or 1..3 (3D)");
  if (!(gamma > 1.0)) return bad("gamma must exceed 1");
  if (!(dt > 0.0)) return bad("dt must be positive");
  if (count < 0) return bad("count must be >= 0");
  if (!h) return bad("h is null");
  for (int k = 0; k < dim; ++k)
    if (!(h[k] > 0.0)) return bad("subcell widths must be positive");
  if (count > 0 && (!patches || !vnew)) return bad("patches and vnew must be device pointers");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return bad("no device");
  unsigned char* base;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_device_base[dev]) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) {
        if (err && errlen)
          snprintf(err, errlen, "cudaGetSymbolAddress of the static scratch failed: %s",
                   cudaGetErrorString(e));
        return ADG_ERR_CUDA;
      }
      g_device_base[dev] = static_cast<unsigned char*>(ptr);
    }
    base = g_device_base[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (dim == 2) {
    switch (N) {
      case 1: return run_noalloc<2, 1>(base, gamma, h, dt, patches, count, vnew, faces, s, err, errlen);
      case 2: return run_noalloc<2, 2>(base, gamma, h, dt, patches, count, vnew, faces, s, err, errlen);
      case 3: return run_noalloc<2, 3>(base, gamma, h, dt, patches, count, vnew, faces, s, err, errlen);
      case 4: return run_noalloc<2, 4>(base, gamma, h, dt, patches, count, vnew, faces, s, err, errlen);
      case 5: return run_noalloc<2, 5>(base, gamma, h, dt, patches, count, vnew, faces, s, err, errlen);
      case 6: return run_noalloc<2, 6>(base, gamma, h, dt, patches, count, vnew, faces, s, err, errlen);
      case 7: return run_noalloc<2, 7>(base, gamma, h, dt, patches, count, vnew, faces, s, err, errlen);
      case 8: return run_noalloc<2, 8>(base, gamma, h, dt, patches, count, vnew, faces, s, err, errlen);
      case 9: return run_noalloc<2, 9>(base, gamma, h, dt, patches, count, vnew, faces, s, err, errlen);
    }
  } else {
    switch (N) {
      case 1: return run_noalloc<3, 1>(base, gamma, h, dt, patches, count, vnew, faces, s, err, errlen);
      case 2: return run_noalloc<3, 2>(base, gamma, h, dt, patches, count, vnew, faces, s, err, errlen);
      case 3: return run_noalloc<3, 3>(base, gamma, h, dt, patches, count, vnew, faces, s, err, errlen);
    }
  }
  return bad("unsupported degree");
}
