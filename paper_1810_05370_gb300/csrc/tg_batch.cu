// tg_batch.cu -- batched solves for many simulations of different grid sizes.
//
// Every simulation of a batch is cut into the same kind of work items: grid tiles of
// BX x BY x zc nodes for stencil work and flat ranges of FLAT_GROUPS float4 groups for vector
// updates.  The tiles of all simulations form one list (likewise the flat ranges), so one
// launch covers the whole batch.  The iterative solves run in persistent cooperative kernels:
// a grid of co-resident blocks walks the lists phase by phase, with a grid-wide barrier
// between phases, and keeps iterating until every simulation's CG has stopped.  Each
// simulation keeps its own CG scalars; its partial sums are combined, in a fixed order, by the
// last of its items to finish (reduce_indexed), so converged simulations simply drop out.
//
// The barrier is a counter plus a generation word.  Its waits read %globaltimer and give up
// after timeout_ns, setting an error flag that makes every block return at its next barrier;
// the host reports TG_ERR_TIMEOUT.  Co-residency is guaranteed by the cooperative launch.
#include "tg_tiles.cuh"

namespace tg {
namespace {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ bool grid_barrier(const BatchDev& B) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    volatile unsigned int* gen = B.bar + 1;
    volatile int* err = B.err;
    const unsigned int g = *gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(B.bar, 1u) + 1u;
    int good = 1;
    if (arrived == gridDim.x) {
      atomicExch(B.bar, 0u);
      __threadfence();
      atomicAdd(B.bar + 1, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*gen == g) {
        if (*err) {
          good = 0;
          break;
        }
        if (global_ns() - t0 > B.timeout_ns) {
          atomicExch(B.err, 1);
          good = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok = good && (*err == 0);
  }
  __syncthreads();
  return ok;
}

__device__ __forceinline__ int ld_status(const CgScal* S) {
  return *(volatile const int*)&S->status;
}

__device__ __forceinline__ void tile_coords(const BSim& S, int local, int& bx, int& by, int& bz) {
  const int gx = S.G.grid.x, gy = S.G.grid.y;
  bx = local % gx;
  by = (local / gx) % gy;
  bz = local / (gx * gy);
}

// ------------------------------------------------------------------------------ resets, status

__global__ void k_batch_reset(BatchDev B) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B.nsims) return;
  const BSim& S = B.sims[s];
  CgScal o = {};
  o.rtol = S.rtol_elas;
  o.maxit = S.maxit_elas;
  o.status = CG_RUNNING;
  *S.Sout = o;
  for (int r = 0; r < 3; ++r) {
    CgScal c = {};
    c.rtol = S.rtol_diff;
    c.maxit = S.maxit_diff;
    c.status = CG_RUNNING;
    S.C.S[r] = c;
  }
  *S.C.counter = 0u;
}

// for timing only: make every inner solve run (tolerance 0) whatever its residual is
__global__ void k_batch_force_inner(BatchDev B) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B.nsims) return;
  CgScal* S = B.sims[s].I.S;
  S->status = CG_RUNNING;
  S->rtol = 0.0;
  S->maxit = 1 << 30;
}

// per simulation: outer elasticity status, residual count, inner iterations, CN statuses and
// iterations, relative residuals
__global__ void k_batch_status(BatchDev B, BatchStat* out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B.nsims) return;
  const BSim& S = B.sims[s];
  BatchStat b;
  b.elas_status = S.Sout->status;
  b.elas_sweeps = S.Sout->it;
  b.elas_inner = S.Sout->pad;
  b.elas_relres = S.Sout->bb > 0.0 ? sqrt(S.Sout->rr / S.Sout->bb) : 0.0;
  for (int r = 0; r < 3; ++r) {
    b.cn_status[r] = S.C.S[r].status;
    b.cn_it[r] = S.C.S[r].it;
    b.cn_relres[r] = S.C.S[r].bb > 0.0 ? sqrt(S.C.S[r].rr / S.C.S[r].bb) : 0.0;
  }
  out[s] = b;
}

// ------------------------------------------------------------------------------ diffusion

__global__ void __launch_bounds__(NT) k_batch_cn_init(BatchDev B) {
  const int t = blockIdx.x;
  const BSim& S = B.sims[B.tile_sim[t]];
  const int local = t - S.tile0;
  int bx, by, bz;
  tile_coords(S, local, bx, by, bz);
  double acc[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) acc[q] = 0.0;
  cn_init_tile(S.G, S.C, bx, by, bz, acc);
  double out[9];
  if (reduce_indexed<9>(acc, S.C.partial, S.C.counter, local, S.ntiles, out) && threadIdx.x == 0 &&
      threadIdx.y == 0) {
#pragma unroll
    for (int r = 0; r < 3; ++r) cg_after_init(S.C.S[r], out[3 * r], out[3 * r + 1], out[3 * r + 2]);
  }
}

__global__ void __launch_bounds__(NT) k_batch_cn_solve(BatchDev B) {
  for (int iter = 0; iter <= B.maxit; ++iter) {
    bool any = false;
    for (int s = 0; s < B.nsims && !any; ++s)
      for (int r = 0; r < 3; ++r) any |= ld_status(&B.sims[s].C.S[r]) == CG_RUNNING;
    if (!any) return;
    // q = A p
    for (int t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
      const BSim& S = B.sims[B.tile_sim[t]];
      bool act[3], a_any = false;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        act[r] = ld_status(&S.C.S[r]) == CG_RUNNING;
        a_any |= act[r];
      }
      if (!a_any) continue;
      const int local = t - S.tile0;
      int bx, by, bz;
      tile_coords(S, local, bx, by, bz);
      double acc[3] = {0.0, 0.0, 0.0};
      cn_matvec_tile<true>(S.G, S.C, act, bx, by, bz, acc);
      double out[3];
      if (reduce_indexed<3>(acc, S.C.partial, S.C.counter, local, S.ntiles, out) &&
          threadIdx.x == 0 && threadIdx.y == 0) {
#pragma unroll
        for (int r = 0; r < 3; ++r)
          if (act[r]) {
            CgScal c = ld_cg(&S.C.S[r]);
            c.pq = out[r];
            c.alpha = c.rz / out[r];
            st_cg(&S.C.S[r], c);
          }
      }
    }
    if (!grid_barrier(B)) return;
    // x += alpha p, r -= alpha q
    for (int t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
      const BSim& S = B.sims[B.tile_sim[t]];
      bool act[3], a_any = false;
      double alpha[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        act[r] = ld_status(&S.C.S[r]) == CG_RUNNING;
        alpha[r] = *(volatile const double*)&S.C.S[r].alpha;
        a_any |= act[r];
      }
      if (!a_any) continue;
      const int local = t - S.tile0;
      int bx, by, bz;
      tile_coords(S, local, bx, by, bz);
      double acc[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) acc[q] = 0.0;
      cn_update_tile(S.G, S.C, act, alpha, bx, by, bz, acc);
      double out[6];
      if (reduce_indexed<6>(acc, S.C.partial, S.C.counter, local, S.ntiles, out) &&
          threadIdx.x == 0 && threadIdx.y == 0) {
#pragma unroll
        for (int r = 0; r < 3; ++r)
          if (act[r]) {
            CgScal c = ld_cg(&S.C.S[r]);
            cg_after_update(c, out[2 * r], out[2 * r + 1]);
            st_cg(&S.C.S[r], c);
          }
      }
    }
    if (!grid_barrier(B)) return;
    // p = D^{-1} r + beta p
    for (int t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
      const BSim& S = B.sims[B.tile_sim[t]];
      bool act[3], a_any = false;
      double beta[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        act[r] = ld_status(&S.C.S[r]) == CG_RUNNING;
        beta[r] = *(volatile const double*)&S.C.S[r].beta;
        a_any |= act[r];
      }
      if (!a_any) continue;
      int bx, by, bz;
      tile_coords(S, t - S.tile0, bx, by, bz);
      cn_pupdate_tile(S.G, S.C, act, beta, bx, by, bz);
    }
    if (!grid_barrier(B)) return;
  }
}

// ------------------------------------------------------------------------------ elasticity

__global__ void __launch_bounds__(NT) k_batch_ir_residual(BatchDev B) {
  const int t = blockIdx.x;
  const BSim& S = B.sims[B.tile_sim[t]];
  if (ld_status(S.Sout) != CG_RUNNING) return;
  const int local = t - S.tile0;
  int bx, by, bz;
  tile_coords(S, local, bx, by, bz);
  double acc[3] = {0.0, 0.0, 0.0};
  elas_ir_residual_tile(S.G, S.E, S.I, 1, bx, by, bz, acc);
  double out[3];
  if (reduce_indexed<3>(acc, S.E.partial, S.E.counter, local, S.ntiles, out) && threadIdx.x == 0 &&
      threadIdx.y == 0)
    elas_ir_residual_finalize(*S.Sout, *S.I.S, out[0], out[1], out[2], B.tau_min, B.max_sweeps);
}

__global__ void __launch_bounds__(NT, 4) k_batch_elas_inner(BatchDev B) {
  __shared__ Tile32 T;
  for (int iter = 0; iter <= B.maxit; ++iter) {
    bool any = false;
    for (int s = 0; s < B.nsims && !any; ++s) any |= ld_status(B.sims[s].I.S) == CG_RUNNING;
    if (!any) return;
    // operator with the fused p-update
    for (int t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
      const BSim& S = B.sims[B.tile_sim[t]];
      if (ld_status(S.I.S) != CG_RUNNING) continue;
      const int local = t - S.tile0;
      int bx, by, bz;
      tile_coords(S, local, bx, by, bz);
      const int it = *(volatile const int*)&S.I.S->it;
      const double beta = *(volatile const double*)&S.I.S->beta;
      const float part = elas32_matvec_tile<true>(S.G, S.K, S.I, it, beta, bx, by, bz, T);
      double acc[1] = {(double)part};
      double out[1];
      if (reduce_indexed<1>(acc, S.I.partial, S.I.counter, local, S.ntiles, out) &&
          threadIdx.x == 0 && threadIdx.y == 0) {
        CgScal c = ld_cg(S.I.S);
        c.pq = out[0];
        c.alpha = c.rz / out[0];
        st_cg(S.I.S, c);
      }
    }
    if (!grid_barrier(B)) return;
    // e += alpha p, r -= alpha q
    for (int t = blockIdx.x; t < B.nitems; t += gridDim.x) {
      const BSim& S = B.sims[B.item_sim[t]];
      if (ld_status(S.I.S) != CG_RUNNING) continue;
      const int local = t - S.item0;
      const float alpha = (float)*(volatile const double*)&S.I.S->alpha;
      const int pb = ((*(volatile const int*)&S.I.S->it) & 1) ^ 1;
      const long long n4 = S.n / 4;
      const long long g0 = (long long)local * FLAT_GROUPS;
      const long long g1 = g0 + FLAT_GROUPS < n4 ? g0 + FLAT_GROUPS : n4;
      const int tid = threadIdx.y * blockDim.x + threadIdx.x;
      double drz = 0.0, drr = 0.0;
      elas32_update_range<true>(S.I, S.n, g0 + tid, g1, NT, alpha, pb, local == S.nitems - 1,
                                drz, drr);
      double acc[2] = {drz, drr};
      double out[2];
      if (reduce_indexed<2>(acc, S.I.partial, S.I.counter, local, S.nitems, out) &&
          threadIdx.x == 0 && threadIdx.y == 0) {
        CgScal c = ld_cg(S.I.S);
        cg_after_update(c, out[0], out[1]);
        st_cg(S.I.S, c);
      }
    }
    if (!grid_barrier(B)) return;
  }
}

__global__ void __launch_bounds__(NT) k_batch_ir_correct(BatchDev B) {
  const int t = blockIdx.x;
  const BSim& S = B.sims[B.item_sim[t]];
  if (ld_status(S.Sout) != CG_RUNNING) return;
  const int local = t - S.item0;
  const long long c0 = (long long)local * FLAT_GROUPS * 4;
  const long long c1 = (local == S.nitems - 1) ? S.n : c0 + FLAT_GROUPS * 4;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  elas_ir_correct_range(S.E, S.I, c0 + tid, c1, NT);
}

// v = du / dt (u = 0 where the right-hand side vanished)
__global__ void __launch_bounds__(NT) k_batch_ir_finish(BatchDev B, double inv_dt) {
  const int t = blockIdx.x;
  const BSim& S = B.sims[B.item_sim[t]];
  const bool zero = ld_status(S.Sout) == CG_ZERO_RHS;
  const int local = t - S.item0;
  const long long c0 = (long long)local * FLAT_GROUPS * 4;
  const long long c1 = (local == S.nitems - 1) ? S.n : c0 + FLAT_GROUPS * 4;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (long long c = c0 + tid; c < c1; c += NT) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double du = S.E.du[a][c];
      if (zero) {
        du -= S.E.u[a][c];
        S.E.u[a][c] = 0.0;
      }
      S.E.v[a][c] = du * inv_dt;
    }
  }
}

cudaError_t launch_coop(const void* fn, int blocks, BatchDev B, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(BX, BY);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[1] = {&B};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace

int batch_coop_blocks_per_sm(int which) {
  int n = 0;
  const void* fn = which == 0 ? (const void*)k_batch_cn_solve : (const void*)k_batch_elas_inner;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, NT, 0) != cudaSuccess) return 0;
  return n;
}

cudaError_t launch_batch_reset(const BatchDev& B, cudaStream_t st) {
  k_batch_reset<<<(B.nsims + 63) / 64, 64, 0, st>>>(B);
  return cudaGetLastError();
}

cudaError_t launch_batch_status(const BatchDev& B, BatchStat* out, cudaStream_t st) {
  k_batch_status<<<(B.nsims + 63) / 64, 64, 0, st>>>(B, out);
  return cudaGetLastError();
}

cudaError_t launch_batch_cn(const BatchDev& B, int coop_blocks, cudaStream_t st) {
  k_batch_cn_init<<<B.ntiles, dim3(BX, BY), 0, st>>>(B);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_coop((const void*)k_batch_cn_solve, coop_blocks, B, st);
}

cudaError_t launch_batch_sweep(const BatchDev& B, int coop_blocks, cudaStream_t st) {
  k_batch_ir_residual<<<B.ntiles, dim3(BX, BY), 0, st>>>(B);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_coop((const void*)k_batch_elas_inner, coop_blocks, B, st);
  if (e != cudaSuccess) return e;
  k_batch_ir_correct<<<B.nitems, dim3(BX, BY), 0, st>>>(B);
  return cudaGetLastError();
}

cudaError_t launch_batch_elas_inner(const BatchDev& B, int coop_blocks, cudaStream_t st) {
  return launch_coop((const void*)k_batch_elas_inner, coop_blocks, B, st);
}

cudaError_t launch_batch_residual(const BatchDev& B, cudaStream_t st) {
  k_batch_ir_residual<<<B.ntiles, dim3(BX, BY), 0, st>>>(B);
  return cudaGetLastError();
}

cudaError_t launch_batch_force_inner(const BatchDev& B, cudaStream_t st) {
  k_batch_force_inner<<<(B.nsims + 63) / 64, 64, 0, st>>>(B);
  return cudaGetLastError();
}

cudaError_t launch_batch_finish(const BatchDev& B, double inv_dt, cudaStream_t st) {
  k_batch_ir_finish<<<B.nitems, dim3(BX, BY), 0, st>>>(B, inv_dt);
  return cudaGetLastError();
}

}  // namespace tg
