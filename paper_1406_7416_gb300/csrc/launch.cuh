// Launch configuration of every kernel for one (dimension, degree).
#pragma once

#include "kernels_misc.cuh"
#include "kernels_pred.cuh"

namespace adg {

constexpr int kBlocksPerSM = 8;
constexpr int kNumSM = 152;

inline int grid_for(long long work, int threads, int cap_blocks = kNumSM * kBlocksPerSM * 4) {
  long long b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap_blocks) b = cap_blocks;
  return (int)b;
}

inline int cells_grid(long long cells) {
  return (int)(cells < (1LL << 30) ? cells : (1LL << 30));
}

// Multiprocessors of the current device (queried once).
inline int device_sms() {
  static int sms = [] {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
      cudaGetLastError();
      return kNumSM;
    }
    return n;
  }();
  return sms;
}

// Grid of a persistent kernel: the blocks that fit on the device at once (at
// least one per multiprocessor), at most `work` blocks.
template <typename K>
int persistent_grid(K kernel, int threads, size_t smem, long long work) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  if (per_sm < 1) per_sm = 1;
  long long g = (long long)per_sm * device_sms();
  if (g > work) g = work;
  if (g < 1) g = 1;
  return (int)g;
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Copy the FP32 Picard operators of degree N into this translation unit's
// constant memory (static: every unit that launches the predictor has its own).
static inline cudaError_t upload_picard_constants_here(int N, const Ops& o) {
  const int n = N + 1;
  cudaError_t e = cudaMemcpyToSymbol(c_Dmf, o.Df, sizeof(float) * n * n,
                                     sizeof(float) * (size_t)N * MAXN * MAXN);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_Ktf, o.Ktf, sizeof(float) * n * n, sizeof(float) * (size_t)N * MAXN * MAXN);
  if (e != cudaSuccess) return e;
  float d3[9], k3[9];
  for (int i = 0; i < 9; ++i) {
    d3[i] = (float)o.D3[i];
    k3[i] = (float)o.Kt3[i];
  }
  e = cudaMemcpyToSymbol(c_D3f, d3, sizeof(d3));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_K3f, k3, sizeof(k3));
}

template <int D, int N>
struct Launch {
  using DM = Dims<D, N>;
  static constexpr int n = DM::n, NV = DM::NV, ND = DM::ND, NSD = DM::NSD, Ns = DM::Ns;

  template <bool MIXED>
  static int pred_threads() {
    int t = ((NV * DM::NST + 31) / 32) * 32;
    return t > PredShape<D, N, MIXED>::threads ? PredShape<D, N, MIXED>::threads : t;
  }
  static size_t cell_smem() { return (size_t)(2 * NV * NSD + 2 * Ns * n + 4 * NV + 128) * sizeof(double); }
  static size_t fallback_smem() {
    constexpr size_t NE = Ns + 2, NB = (D == 3) ? NE * NE * NE : NE * NE;
    return (size_t)(NV * NB + 2 * NV * NSD + NV * (Ns + 1) * DM::NSF + 2 * Ns * n + 2 * NV + 128) *
           sizeof(double);
  }
  static size_t fix_smem() {
    return (size_t)(NV * ND + 2 * NV * NSD + 2 * Ns * n + 4 * NV + 128) * sizeof(double);
  }

  // (an event node when the stream is being captured into a graph)
  static void mark(cudaEvent_t* ev, int phase, cudaStream_t s) {
    if (!ev) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
      cudaEventRecordWithFlags(ev[phase], s, cudaEventRecordExternal);
    else
      cudaEventRecord(ev[phase], s);
  }

  // the warp-per-cell predictor exists for the degrees whose mixed default
  // is the split final stage (2D N <= 5, 3D)
  static constexpr bool kSplit = !(D == 2 && N >= 6);

  template <int W, bool TC>
  static cudaError_t launch_split(const Batch& cells, long long total, cudaStream_t s) {
    if constexpr (kSplit) {
      const size_t sm = split_smem_bytes<D, N, W>();
      cudaError_t e = set_smem(k_predictor_split<D, N, W, TC>, sm);
      if (e != cudaSuccess) return e;
      static const int grid_full = persistent_grid(k_predictor_split<D, N, W, TC>, 32 * W, sm, 1LL << 40);
      const long long groups = (total + W - 1) / W;
      const int grid = (int)(groups < grid_full ? groups : grid_full);
      k_predictor_split<D, N, W, TC><<<grid, 32 * W, sm, s>>>(cells);
      return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
  }

  // The predictor in the launch shape sl.pred (PRED_*); shapes that do not
  // apply to the launch fall back to the block-per-cell kernel.
  static cudaError_t launch_predictor(const StepLaunch& sl, cudaStream_t s) {
    cudaError_t e;
    const int grid = cells_grid(sl.total_cells);
    const Batch cells{sl.pps, sl.n, sl.pre_cells};
    if (sl.prec == ADG_PREC_MIXED_FP32) {
      if (kSplit && sl.pred == PRED_WARP1) return launch_split<1, false>(cells, sl.total_cells, s);
      if (kSplit && sl.pred == PRED_WARP2) return launch_split<2, false>(cells, sl.total_cells, s);
      if (kSplit && sl.pred == PRED_WARP4) return launch_split<4, false>(cells, sl.total_cells, s);
      if (kSplit && sl.pred == PRED_WARP4_TC) return launch_split<4, true>(cells, sl.total_cells, s);
      const size_t sm = predictor_smem_bytes<D, N, true>();
      if ((e = set_smem(k_predictor<D, N, true>, sm)) != cudaSuccess) return e;
      const bool alt = sl.pred == PRED_BLOCK_ALT;
      const int th = alt ? alt_threads<true>() : pred_threads<true>();
      static const int gp = persistent_grid(k_predictor<D, N, true>, pred_threads<true>(), sm, 1LL << 40);
      static const int ga = persistent_grid(k_predictor<D, N, true>, alt_threads<true>(), sm, 1LL << 40);
      const int gmax = alt ? ga : gp;
      k_predictor<D, N, true><<<grid < gmax ? grid : gmax, th, sm, s>>>(cells);
    } else {
      const size_t sm = predictor_smem_bytes<D, N, false>();
      if ((e = set_smem(k_predictor<D, N, false>, sm)) != cudaSuccess) return e;
      const bool alt = sl.pred == PRED_BLOCK_ALT;
      const int th = alt ? alt_threads<false>() : pred_threads<false>();
      static const int gn = persistent_grid(k_predictor<D, N, false>, pred_threads<false>(), sm, 1LL << 40);
      static const int ga = persistent_grid(k_predictor<D, N, false>, alt_threads<false>(), sm, 1LL << 40);
      const int gmax = alt ? ga : gn;
      k_predictor<D, N, false><<<grid < gmax ? grid : gmax, th, sm, s>>>(cells);
    }
    return cudaGetLastError();
  }

  // The other block width of the block-per-cell predictor (PRED_BLOCK_ALT):
  // 256 threads where the default is below its launch bound of 256 (fewer when
  // a cell has fewer work items), 128 where the default is 256, and 64 where
  // the default is the kernel's launch bound.  Every width computes the same
  // outputs (each work item's arithmetic does not depend on the width).
  template <bool MIXED>
  static int alt_threads() {
    const int def = pred_threads<MIXED>();
    const int bound = PredShape<D, N, MIXED>::bound;
    if (def >= 256) return 128;
    if (bound >= 256) {
      const int t = ((NV * DM::NST + 31) / 32) * 32;
      return t > 256 ? 256 : t;
    }
    return 64;
  }

  static cudaError_t step_dg(const StepLaunch& sl, cudaStream_t s) {
    cudaError_t e;
    cudaEvent_t* ev = sl.ev;
    if (sl.total_cells == 0) return cudaSuccess;
    const int grid = cells_grid(sl.total_cells);
    const Batch cells{sl.pps, sl.n, sl.pre_cells};
    mark(ev, PHASE_PREDICTOR, s);
    if ((e = launch_predictor(sl, s)) != cudaSuccess) return e;
    mark(ev, PHASE_FACEFLUX, s);
    for (int k = 0; k < D; ++k) {
      const Batch faces{sl.pps, sl.n, sl.pre_faces[k]};
      k_faceflux<D, N><<<grid_for(sl.total_faces[k], 256), 256, 0, s>>>(faces, k);
    }
    mark(ev, PHASE_CORRECT, s);
    if constexpr (D == 2) {
      // one warp per cell, CD_WARPS cells per block, persistent over the cells
      const size_t sc = correct_warp_smem_bytes<D, N>();
      if ((e = set_smem(k_correct_detect_w<D, N>, sc)) != cudaSuccess) return e;
      static const int grid_cd = persistent_grid(k_correct_detect_w<D, N>, 32 * CD_WARPS, sc, 1LL << 40);
      const long long groups = (sl.total_cells + CD_WARPS - 1) / CD_WARPS;
      k_correct_detect_w<D, N><<<(int)(groups < grid_cd ? groups : grid_cd), 32 * CD_WARPS, sc, s>>>(cells);
    } else {
      // 3D: a cell's subcell data (Ns^3 per variable) fills a block's shared
      // memory, and four warps per cell hide its latency better
      const size_t sc = correct_smem_bytes<D, N>();
      if ((e = set_smem(k_correct_detect<D, N>, sc)) != cudaSuccess) return e;
      static const int grid_cd = persistent_grid(k_correct_detect<D, N>, 128, sc, 1LL << 40);
      k_correct_detect<D, N><<<(int)(sl.total_cells < grid_cd ? sl.total_cells : grid_cd), 128, sc, s>>>(cells);
    }
    return cudaGetLastError();
  }

  // One limiter pass (pass < 0: the pass of the device-sized loop).
  static cudaError_t lim_pass(const StepLaunch& sl, int pass, cudaStream_t s) {
    cudaError_t e;
    constexpr int SPB = (D == 2) ? SUBS_PER_BLOCK_2D : SUBS_PER_BLOCK_3D;
    const Batch lim{sl.pps, sl.n, sl.pre_lim};
    const long long ch = sl.sum_chunk;    // upper bound of the troubled cells of one pass
    if ((e = launch_lim_prefix(sl, pass, s)) != cudaSuccess) return e;
    k_lim_patch<D, N><<<grid_for(ch * ipow(3, D), 1, kNumSM * 16), 128, 0, s>>>(lim, pass);
    const long long ncross = ch * (DM::NSD + 2 * D * DM::NSF);
    const int gs = grid_for(ch * NV * DM::LD, 256), gp = grid_for(ncross, SPB, kNumSM * 16);
    // the subcell predictor stored in FP32 when it runs wholly in FP32
    const bool qf = sl.prec == ADG_PREC_MIXED_FP32 && sl.sub_f32 && sl.sub32 == 3;
    // register form with the Rusanov sub-face flux: the predictor leaves face
    // traces (SubTraces2 / SubTraces) for k_lim_flux_t2 / k_lim_flux_t instead
    // of nodal values
    const bool traces = qf && sl.sub_reg && sl.flux == ADG_FLUX_RUSANOV;
    if (sl.prec == ADG_PREC_MIXED_FP32 && sl.sub_f32) {
      // mixed precision: FP32 reconstruction feeding the FP32 subcell predictor
      k_lim_sweep<D, N, 0, float><<<gs, 256, 0, s>>>(lim, pass);
      k_lim_sweep<D, N, 1, float><<<gs, 256, 0, s>>>(lim, pass);
      if (D == 3) k_lim_sweep<D, N, (D == 3 ? 2 : 1), float><<<gs, 256, 0, s>>>(lim, pass);
      if (qf) {
        // one warp per subcell, blocks looping over the pass's subcells; by
        // default the subcell's space-time nodes live in the warp's registers
        if (sl.sub_reg && D == 2) {
          if constexpr (D == 2) {
            static_assert(SubTraces2<N>::per_cell <= 2LL * DM::NED * DM::NV * DM::NST3,
                          "the traces fit the subcell predictor's scratch");
            const long long want = ((ncross + 2) / 3 + 7) / 8;      // three subcells per warp
            if (traces) {
              static const int gw = persistent_grid(k_lim_predict_s2<N, true>, 256, 0, 1LL << 40);
              k_lim_predict_s2<N, true><<<(int)(want < gw ? want : gw), 256, 0, s>>>(lim);
            } else {
              static const int gw = persistent_grid(k_lim_predict_s2<N, false>, 256, 0, 1LL << 40);
              k_lim_predict_s2<N, false><<<(int)(want < gw ? want : gw), 256, 0, s>>>(lim);
            }
          }
        } else if (traces) {
          if constexpr (D == 3) {
            static_assert(SubTraces<N>::per_cell <= 2LL * DM::NED * DM::NV * DM::NST3,
                          "the traces fit the subcell predictor's scratch");
            static const int gw = persistent_grid(k_lim_predict_s3<N>, 256, 0, 1LL << 40);
            const long long want = (ncross + 7) / 8;
            k_lim_predict_s3<N><<<(int)(want < gw ? want : gw), 256, 0, s>>>(lim);
          }
        } else {
          constexpr int W = LimWarps<D>::W;
          static const int gw = persistent_grid(k_lim_predict_w<D, N>, 32 * W, 0, 1LL << 40);
          const long long want = (ncross + W - 1) / W;
          k_lim_predict_w<D, N><<<(int)(want < gw ? want : gw), 32 * W, 0, s>>>(lim);
        }
      } else
        k_lim_predict<D, N, true, float, false><<<gp, SPB * DM::NST3, 0, s>>>(lim, pass, sl.sub32);
    } else {
      k_lim_sweep<D, N, 0, double><<<gs, 256, 0, s>>>(lim, pass);
      k_lim_sweep<D, N, 1, double><<<gs, 256, 0, s>>>(lim, pass);
      if (D == 3) k_lim_sweep<D, N, (D == 3 ? 2 : 1), double><<<gs, 256, 0, s>>>(lim, pass);
      if (sl.prec == ADG_PREC_MIXED_FP32)
        k_lim_predict<D, N, true, double, false><<<gp, SPB * DM::NST3, 0, s>>>(lim, pass, sl.sub32);
      else
        k_lim_predict<D, N, false, double, false><<<gp, SPB * DM::NST3, 0, s>>>(lim, pass, 0);
    }
    const int gf = grid_for(ch * (Ns + 1) * DM::NSF, 256);
    if (traces && D == 2) {
      if constexpr (D == 2) {
        // three sub-faces per warp, persistent
        const long long want = ((ch * (Ns + 1) * DM::NSF + 2) / 3 + 7) / 8;
        static const int g0 = persistent_grid(k_lim_flux_t2<N, 0>, 256, 0, 1LL << 40);
        static const int g1 = persistent_grid(k_lim_flux_t2<N, 1>, 256, 0, 1LL << 40);
        k_lim_flux_t2<N, 0><<<(int)(want < g0 ? want : g0), 256, 0, s>>>(lim, pass);
        k_lim_flux_t2<N, 1><<<(int)(want < g1 ? want : g1), 256, 0, s>>>(lim, pass);
      }
    } else if (traces) {
      if constexpr (D == 3) {
        // one warp per sub-face, persistent
        const long long want = (ch * (Ns + 1) * DM::NSF + 7) / 8;
        static const int g0 = persistent_grid(k_lim_flux_t<N, 0>, 256, 0, 1LL << 40);
        static const int g1 = persistent_grid(k_lim_flux_t<N, 1>, 256, 0, 1LL << 40);
        static const int g2 = persistent_grid(k_lim_flux_t<N, 2>, 256, 0, 1LL << 40);
        k_lim_flux_t<N, 0><<<(int)(want < g0 ? want : g0), 256, 0, s>>>(lim, pass);
        k_lim_flux_t<N, 1><<<(int)(want < g1 ? want : g1), 256, 0, s>>>(lim, pass);
        k_lim_flux_t<N, 2><<<(int)(want < g2 ? want : g2), 256, 0, s>>>(lim, pass);
      }
    } else if (sl.prec == ADG_PREC_MIXED_FP32 && sl.sub_f32 && sl.flux == ADG_FLUX_RUSANOV) {
      if (qf) {
        k_lim_flux<D, N, 0, float, float><<<gf, 256, 0, s>>>(lim, pass);
        k_lim_flux<D, N, 1, float, float><<<gf, 256, 0, s>>>(lim, pass);
        if (D == 3) k_lim_flux<D, N, (D == 3 ? 2 : 1), float, float><<<gf, 256, 0, s>>>(lim, pass);
      } else {
        k_lim_flux<D, N, 0, float, double><<<gf, 256, 0, s>>>(lim, pass);
        k_lim_flux<D, N, 1, float, double><<<gf, 256, 0, s>>>(lim, pass);
        if (D == 3) k_lim_flux<D, N, (D == 3 ? 2 : 1), float, double><<<gf, 256, 0, s>>>(lim, pass);
      }
    } else if (qf) {
      k_lim_flux<D, N, 0, double, float><<<gf, 256, 0, s>>>(lim, pass);
      k_lim_flux<D, N, 1, double, float><<<gf, 256, 0, s>>>(lim, pass);
      if (D == 3) k_lim_flux<D, N, (D == 3 ? 2 : 1), double, float><<<gf, 256, 0, s>>>(lim, pass);
    } else {
      k_lim_flux<D, N, 0, double, double><<<gf, 256, 0, s>>>(lim, pass);
      k_lim_flux<D, N, 1, double, double><<<gf, 256, 0, s>>>(lim, pass);
      if (D == 3) k_lim_flux<D, N, (D == 3 ? 2 : 1), double, double><<<gf, 256, 0, s>>>(lim, pass);
    }
    k_lim_update<D, N><<<(int)(ch < kNumSM * 8 ? ch : kNumSM * 8), 128, cell_smem(), s>>>(lim, pass);
    return cudaGetLastError();
  }

  // The limiter passes as a conditional WHILE node of the graph being
  // captured on `s`: the body (one pass on the device-stored pass index, then
  // k_lim_loop_next) is captured into the node's child graph on sl.body.
  static cudaError_t lim_loop(const StepLaunch& sl, cudaStream_t s) {
    cudaError_t e;
    if ((e = launch_lim_loop_begin(sl, s)) != cudaSuccess) return e;
    cudaGraph_t body = nullptr;
    if ((e = add_loop_node(s, sl.cond, &body)) != cudaSuccess) return e;
    if ((e = cudaStreamBeginCaptureToGraph(sl.body, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return e;
    e = lim_pass(sl, -1, sl.body);
    if (e == cudaSuccess) e = launch_lim_loop_next(sl, sl.body);
    cudaGraph_t captured = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(sl.body, &captured);
    return e != cudaSuccess ? e : ee;
  }

  static cudaError_t step_limiter(const StepLaunch& sl, cudaStream_t s) {
    cudaError_t e;
    cudaEvent_t* ev = sl.ev;
    mark(ev, PHASE_LIMITER, s);
    const size_t su = cell_smem();
    if ((e = set_smem(k_lim_update<D, N>, su)) != cudaSuccess) return e;
    if (sl.loop) {
      if ((e = lim_loop(sl, s)) != cudaSuccess) return e;
    } else {
      for (int pass = 0; pass < sl.max_passes; ++pass)
        if ((e = lim_pass(sl, pass, s)) != cudaSuccess) return e;
    }
    if (sl.cascade) {
      // first-order layer after WENO3 (Sec. 6, Fig. algo2); both lists are
      // empty in most steps and the kernels then return at once
      if ((e = launch_count_prefix(sl, sl.pre_fb, CNT_FB, s)) != cudaSuccess) return e;
      const size_t sfb = fallback_smem();
      if ((e = set_smem(k_lim_fallback<D, N>, sfb)) != cudaSuccess) return e;
      k_lim_fallback<D, N><<<kNumSM, 128, sfb, s>>>(Batch{sl.pps, sl.n, sl.pre_fb});
      if ((e = launch_count_prefix(sl, sl.pre_refix, CNT_REFIX, s)) != cudaSuccess) return e;
      if ((e = set_smem(k_lim_refix<D, N>, su)) != cudaSuccess) return e;
      k_lim_refix<D, N><<<kNumSM, 128, su, s>>>(Batch{sl.pps, sl.n, sl.pre_refix});
    }
    mark(ev, PHASE_FIX, s);
    if ((e = launch_fix_prefix(sl, s)) != cudaSuccess) return e;
    const size_t sf = fix_smem();
    if ((e = set_smem(k_lim_fix<D, N>, sf)) != cudaSuccess) return e;
    const Batch fix{sl.pps, sl.n, sl.pre_fix};
    k_lim_fix<D, N><<<kNumSM * 8, 128, sf, s>>>(fix);
    mark(ev, PHASE_END, s);
    return cudaGetLastError();
  }

  static cudaError_t run(const LaunchArgs& a) {
    if (a.op == OP_STEP_DG || a.op == OP_STEP_LIMITER) {
      if (a.op == OP_STEP_DG) return step_dg(*a.step, a.stream);
      return step_limiter(*a.step, a.stream);
    }
    if (a.op == OP_PREDICTOR) return a.step->total_cells ? launch_predictor(*a.step, a.stream) : cudaSuccess;
    const Params& p = *a.p;
    cudaStream_t s = a.stream;
    cudaError_t e;
    const int grid = cells_grid(p.geo.cells);
    switch (a.op) {
      case OP_STEP_DG:
        return step_dg(*a.step, s);
      case OP_STEP_LIMITER:
        return step_limiter(*a.step, s);
      case OP_LOAD_DETECT: {
        const size_t sm = cell_smem();
        if ((e = set_smem(k_load_detect<D, N>, sm)) != cudaSuccess) return e;
        k_load_detect<D, N><<<grid, 128, sm, s>>>(p, a.exact, a.cmm_ex);
        return cudaGetLastError();
      }
      case OP_LOAD_FULL: {
        const size_t sm = cell_smem();
        if ((e = set_smem(k_load_full<D, N>, sm)) != cudaSuccess) return e;
        k_load_full<D, N><<<grid, 128, sm, s>>>(p, a.beta, a.sub);
        return cudaGetLastError();
      }
      case OP_READ_FULL:
        k_read_full<D, N><<<grid_for(p.geo.cells * NV * NSD, 256), 256, 0, s>>>(p, a.out);
        return cudaGetLastError();
      case OP_PROJECT:
        k_project<D, N><<<grid, 128, 0, s>>>(p, *a.prob, a.fac, a.out);
        return cudaGetLastError();
      case OP_LAMBDA: {
        const size_t sm = cell_smem();
        if ((e = set_smem(k_lambda<D, N>, sm)) != cudaSuccess) return e;
        k_lambda<D, N><<<grid, 128, sm, s>>>(p);
        return cudaGetLastError();
      }
      case OP_PACK:
      case OP_UNPACK: {
        Box bx;
        bx.count = 1;
        for (int k = 0; k < 3; ++k) {
          bx.lo[k] = k < D ? a.box[k] : 0;
          bx.hi[k] = k < D ? a.box[3 + k] : 1;
          bx.count *= bx.hi[k] - bx.lo[k];
        }
        const int gb = (int)(bx.count < kNumSM * 8 ? bx.count : kNumSM * 8);
        if (a.op == OP_PACK) {
          k_pack<D, N><<<gb, 128, 0, s>>>(p, bx, a.buf);
          return cudaGetLastError();
        }
        k_unpack<D, N><<<gb, 128, 0, s>>>(p, bx, a.buf);
        if ((e = cudaMemsetAsync(p.b.counters + CNT_TROUBLED0 + (1 - p.cur), 0, sizeof(int), s)) !=
            cudaSuccess)
          return e;
        k_relist<D, N><<<cells_grid(p.geo.cells < kNumSM * 64 ? p.geo.cells : kNumSM * 64), 128, 0, s>>>(
            p, bx, a.buf);
        k_copyback<D, N><<<kNumSM * 4, 256, 0, s>>>(p);
        return cudaGetLastError();
      }
      case OP_SUB_MINMAX:
        k_sub_minmax<D, N><<<grid_for(p.geo.cells * NV, 256), 256, 0, s>>>(a.sub, a.out,
                                                                            p.geo.cells);
        return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
  }
};

// Scratch of the limiter per troubled cell, in doubles.
template <int D, int N>
size_t scratch_of(size_t* patch, size_t* sw0, size_t* sw1, size_t* sw2, size_t* qsub,
                  size_t* fsub) {
  using DM = Dims<D, N>;
  const size_t NV = DM::NV, L = DM::L, NE = DM::NE;
  *patch = NV * DM::LD;
  *sw0 = NV * NE * (D == 3 ? L * L : L) * 3;
  *sw1 = NV * NE * NE * (D == 3 ? L : 1) * 9;
  *sw2 = (D == 3) ? NV * NE * NE * NE * 27 : 0;
  *qsub = (size_t)DM::NED * NV * DM::NST3;
  *fsub = NV * (DM::Ns + 1) * DM::NSF;
  return *patch + *sw0 + *sw1 + *sw2 + *qsub + D * *fsub;
}

}  // namespace adg
