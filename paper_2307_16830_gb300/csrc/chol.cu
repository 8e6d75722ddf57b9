// Numeric sparse Cholesky factorization of M_cond and solves with it.
//
// The factor L of P M_cond P' is stored in supernodes (dense column-major
// blocks, see symbolic.h).  The factorization is multifrontal: a supernode
// adds its children's update matrices into its panel and into its own
// update matrix (extend-add), factors its panel (a dense Cholesky of the
// diagonal block and the scaled rows below it) and subtracts L21 L21' from
// its update matrix, which its parent adds in turn.
//
// All of it runs in ONE persistent kernel over the task graph of
// chol_plan.h: each block takes the next task of the list (an atomic
// counter), waits until the tasks it depends on have set their finished
// flags, runs it, and sets its own flag.  The list is a topological order,
// so the lowest unfinished task any running block holds has all its
// dependencies finished: the blocks always progress, whether or not all of
// them are resident.  Every wait is bounded (2 s of the GPU clock); a wait
// that runs out sets the object's abort flag, every block then stops, and
// the host reports a timeout.  Data another task wrote is read through L2
// (ld.global.cg): L1 is not coherent across SMs.
//
// Task kinds: a group of small supernodes (one block, level by level, one
// warp per supernode), one block supernode (panel and update matrix staged
// in shared memory), and the tiles of a large supernode's front (32 x 32:
// extend-add into a tile, Cholesky of a diagonal tile, triangular solve of
// a tile below it, a tile minus a product of two such tiles).
//
// A pivot that is not above the tolerance (or is NaN) is recorded (the
// smallest column, so the result does not depend on the schedule) and
// replaced by 1 so the arithmetic stays finite; the factorization then
// counts as failed.  The solves run the same way: the forward solve passes
// update vectors up the tree, the backward solve reads the ancestors' solved
// entries.  Every sum has a fixed order: results are bit-reproducible.
#include "chol_internal.h"
#include "chol_plan.h"

#include <algorithm>

namespace acopf {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kPermThreads = 256;
constexpr int T = kCholTile;
static_assert(T == kCholTileEdge, "host plan and kernels agree on the tile edge");
static_assert(kThreads == T * kWarps, "a tile column per warp, rows over the lanes");
// per-warp staging of a small supernode: panel and update matrix,
// h w + (h - w)^2 <= 32 + 31^2 for h <= 32
constexpr int kSmallStage = 1024;
constexpr int kSmallPanel = kCholWarpRows * kCholWarpCols;  // a small supernode's panel
static_assert(kWarps * kSmallPanel <= kCholMaxWidth * kCholMaxWidth, "solve staging holds a group");
constexpr int cmax(int a, int b) { return a > b ? a : b; }
constexpr int kStageDoubles =
    cmax(cmax(kWarps * kSmallStage, kCholBlockDoubles), cmax(3 * T * T + T, kCholMaxWidth * (kCholMaxWidth + 1)));
constexpr int kRelInts = cmax(kWarps * kCholWarpRows, kCholBlockRows);
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

// ---------------------------------------------------------------------------
// plain kernels: permutation and assembly of M_cond into the blocks
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kPermThreads) k_gather(double* __restrict__ out,
                                                         const double* __restrict__ in,
                                                         const int32_t* __restrict__ idx, int n) {
  for (int t = blockIdx.x * kPermThreads + threadIdx.x; t < n; t += gridDim.x * kPermThreads)
    out[t] = in[__ldg(idx + t)];
}

__global__ void __launch_bounds__(kPermThreads) k_scatter(double* __restrict__ out,
                                                          const double* __restrict__ in,
                                                          const int32_t* __restrict__ idx, int n) {
  for (int t = blockIdx.x * kPermThreads + threadIdx.x; t < n; t += gridDim.x * kPermThreads)
    out[__ldg(idx + t)] = in[t];
}

// Lx[amap[k]] = kvals[k] (Lx zeroed before)
__global__ void __launch_bounds__(kPermThreads) k_chol_assemble(double* __restrict__ Lx,
                                                                const int64_t* __restrict__ amap,
                                                                const double* __restrict__ kvals,
                                                                int64_t nnz) {
  for (int64_t k = int64_t(blockIdx.x) * kPermThreads + threadIdx.x; k < nnz;
       k += int64_t(gridDim.x) * kPermThreads)
    Lx[__ldg(amap + k)] = kvals[k];
}

// ---------------------------------------------------------------------------
// task scheduling
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ld_acquire(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int32_t* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long gpu_clock_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits until *flag is set; false when the abort flag is (or gets) set or
// the wait runs past kWaitLimitNs (then it sets the abort flag).
__device__ bool wait_done(const int32_t* flag, int32_t* abort) {
  if (ld_acquire(flag)) return true;
  const unsigned long long t0 = gpu_clock_ns();
  for (unsigned it = 0;; ++it) {
    __nanosleep(it < 32 ? 64 : 256);
    if (ld_acquire(flag)) return true;
    if ((it & 31) == 31) {
      if (ld_acquire(abort)) return false;
      if (gpu_clock_ns() - t0 > kWaitLimitNs) {
        atomicExch(abort, 1);
        return false;
      }
    }
  }
}

// A kernel launched as a programmatic dependent (see launch_early) may run
// out of tasks while the kernel before it is still running: before its
// blocks exit they wait for that kernel's completion, so that the stream's
// next work sees both finished (a no-op for a kernel launched without it).
__device__ __forceinline__ void wait_prior_grid() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ unsigned sm_id() {
  unsigned r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}

// The persistent loop: take the next task, load what none of its
// dependencies write (`pre`, whose result `run` receives), wait for its
// dependencies and those in the other graph (warp 0's lanes each watch some
// of them), run it with the whole block, publish its flag (fence, then a
// release store); with a trace buffer, record the task's times (ready =
// the dependencies seen done).

template <typename Pre, typename Run>
__device__ __forceinline__ void task_loop(const CholTasks& g, int32_t* abort, Pre pre, Run run) {
  __shared__ int s_task, s_ok;
  __shared__ unsigned long long s_t0;
  for (;;) {
    if (threadIdx.x == 0) {
      s_task = ld_acquire(abort) ? g.n : atomicAdd(g.next, 1);
      if (g.trace) s_t0 = gpu_clock_ns();
    }
    __syncthreads();
    const int t = s_task;
    if (t >= g.n) return;
    const int4 tk = __ldg(g.task + t);
    const auto early = pre(tk);
    if (threadIdx.x < 32) {
      bool ok = true;
      const int q1 = __ldg(g.dep_ptr + t + 1);
      for (int q = __ldg(g.dep_ptr + t) + int(threadIdx.x); q < q1 && ok; q += 32)
        ok = wait_done(g.done + __ldg(g.dep + q), abort);
      if (g.xdep_ptr) {
        const int x1 = __ldg(g.xdep_ptr + t + 1);
        for (int q = __ldg(g.xdep_ptr + t) + int(threadIdx.x); q < x1 && ok; q += 32)
          ok = wait_done(g.xdone + __ldg(g.xdep + q), abort);
      }
      ok = __all_sync(0xffffffffu, ok);
      if (threadIdx.x == 0) s_ok = ok;
    }
    __syncthreads();  // orders the block's reads after warp 0's acquires
    if (!s_ok) return;
    const unsigned long long t1 = g.trace && threadIdx.x == 0 ? gpu_clock_ns() : 0ull;
    run(tk, early);
    __syncthreads();  // the block's writes before thread 0's release
    if (threadIdx.x == 0) {
      st_release(g.done + t, 1);
      if (g.trace) {
        long long* r = g.trace + 6 * size_t(t);
        r[0] = tk.x;
        r[1] = tk.y;
        r[2] = (long long)s_t0;
        r[3] = (long long)t1;
        r[4] = (long long)gpu_clock_ns();
        r[5] = sm_id();
      }
    }
  }
}

template <int NT>
__device__ __forceinline__ void group_sync() {
  if constexpr (NT == 32)
    __syncwarp();
  else
    __syncthreads();
}

// ---------------------------------------------------------------------------
// dense pieces of one supernode (panel P of leading dimension h, update
// matrix U of leading dimension m = h - w, both in shared memory)
// ---------------------------------------------------------------------------
// Column by column: every thread takes the same pivot and its reciprocal;
// the trailing entries go NT per round across columns.
// (FP64 is slow on this part: one warp instruction occupies a sub-partition
// for 64 cycles however many lanes are active, so the pivot's reciprocal
// square root, a 400-cycle chain, is computed by one warp and shared.)
template <int NT>
__device__ void factor_panel(double* __restrict__ P, int h, int w, int f, int tid, double tol,
                             int32_t* bad, double* __restrict__ dinv) {
  const int warp = tid >> 5;
  __shared__ double s_rinv;
  for (int k = 0; k < w; ++k) {
    double rinv = 0.0;
    if (warp == 0) {  // nothing else reads the diagonal entry in this step
      double p = P[size_t(k) * h + k];
      if (!(p > tol)) {
        if (tid == 0) atomicMin(bad, f + k);
        p = 1.0;
      }
      rinv = rsqrt(p);
      if (tid == 0) {
        P[size_t(k) * h + k] = p * rinv;
        dinv[f + k] = rinv;
        if constexpr (NT > 32) s_rinv = rinv;
      }
    }
    group_sync<NT>();
    if constexpr (NT > 32) {
      if (warp != 0) rinv = s_rinv;
    }
    for (int i = k + 1 + tid; i < h; i += NT) P[size_t(k) * h + i] *= rinv;
    group_sync<NT>();
    {
      // the trailing panel entries (j, i), j in (k, w), i in [j, h), column
      // by column, NT per round, so every lane has an entry (an FP64 warp
      // instruction costs the same however many lanes are active)
      int j = k + 1, r = tid;  // entry r of column j (row j + r)
      while (j < w && r >= h - j) {
        r -= h - j;
        ++j;
      }
      while (j < w) {
        P[size_t(j) * h + j + r] -= P[size_t(k) * h + j + r] * P[size_t(k) * h + j];
        r += NT;
        while (j < w && r >= h - j) {
          r -= h - j;
          ++j;
        }
      }
    }
    group_sync<NT>();
  }
}

// (i, j) -> the entry `step` positions further on in the column-by-column
// enumeration of an m x m lower triangle (rows j..m-1 of column j)
__device__ __forceinline__ void tri_advance(int& i, int& j, int m, int step) {
  i += step;
  while (j < m && i >= m) {
    i -= m - j - 1;
    ++j;
  }
}

// U -= L21 L21' on the lower triangle: its entries column by column, NT
// consecutive ones per round (thread tid takes entries tid, tid + NT, ...),
// so every lane has an entry (an FP64 warp instruction costs the same
// however many lanes are active; a column per warp left most lanes of the
// short columns idle).
template <int NT>
__device__ void form_update(const double* __restrict__ P, int h, int w, int tid,
                            double* __restrict__ U) {
  const int m = h - w;
  const int total = m * (m + 1) / 2;
  int i = 0, j = 0;  // entry tid of the triangle: column j, row i
  tri_advance(i, j, m, tid);
  for (int e = tid; e < total; e += NT) {
    double acc = 0.0;
    for (int k = 0; k < w; ++k) acc = fma(P[size_t(k) * h + w + i], P[size_t(k) * h + w + j], acc);
    U[size_t(j) * m + i] -= acc;
    tri_advance(i, j, m, NT);
  }
}

// Extend-add of t's children's update matrices, one child at a time: the
// entries in t's columns go to the panel P, the rest to the update matrix
// U.  A child's descriptor (kid_desc: its update rows, row map and update
// matrix offsets) is read one child ahead, so each child costs one round of
// dependent loads; its row map is staged in `srel`, and the lower triangle
// of its update matrix is read NT entries per round, kBatch rounds in
// flight.
template <int NT>
__device__ void extend_add(const CholDev& d, int t, int tid, double* __restrict__ P, int h,
                           int w, double* __restrict__ U, int* __restrict__ srel) {
  constexpr int kBatch = 8;
  const int m = h - w;
  const int q0 = __ldg(d.kid_ptr + t), q1 = __ldg(d.kid_ptr + t + 1);
  int4 next = q0 < q1 ? __ldg(d.kid_desc + q0) : make_int4(0, 0, 0, 0);
  for (int q = q0; q < q1; ++q) {
    const int4 kd = next;  // the child's descriptor, loaded one child ahead
    if (q + 1 < q1) next = __ldg(d.kid_desc + q + 1);
    const int mc = kd.x;
    const double* __restrict__ Uc =
        d.Ux + ((static_cast<int64_t>(kd.w) << 32) | static_cast<uint32_t>(kd.z));
    const int32_t* __restrict__ rel = d.relmap + kd.y;
    const int nl = mc * (mc + 1) / 2;
    int i = 0, j = 0;
    tri_advance(i, j, mc, tid);
    for (int e0 = 0; e0 < nl; e0 += kBatch * NT) {
      double v[kBatch];
      int ii[kBatch], jj[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        ii[u] = i;
        jj[u] = j;
        v[u] = e0 + u * NT + tid < nl ? __ldcg(Uc + size_t(j) * mc + i) : 0.0;
        tri_advance(i, j, mc, NT);
      }
      if (e0 == 0) {  // the row map, staged while the first batch is in flight
        for (int r = tid; r < mc; r += NT) srel[r] = __ldg(rel + r);
        group_sync<NT>();
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        if (e0 + u * NT + tid >= nl) continue;
        const int ri = srel[ii[u]], rj = srel[jj[u]];
        if (rj < w)
          P[size_t(rj) * h + ri] += v[u];
        else
          U[size_t(rj - w) * m + (ri - w)] += v[u];
      }
    }
    group_sync<NT>();
  }
}

// A supernode staged in shared memory (ws: panel then update matrix) by a
// group of NT threads: load, extend-add, factor, update matrix, store.
template <int NT>
__device__ void factor_staged(const CholDev& d, int t, int tid, double tol,
                              double* __restrict__ ws, int* __restrict__ srel) {
  constexpr int kBatch = 8;
  const int f = __ldg(d.sn_first + t), w = __ldg(d.sn_first + t + 1) - f;
  const int h = __ldg(d.sn_rowptr + t + 1) - __ldg(d.sn_rowptr + t), m = h - w;
  double* __restrict__ Lt = d.Lx + __ldg(d.sn_off + t);
  double* __restrict__ Ut = d.Ux + __ldg(d.u_off + t);
  double* __restrict__ P = ws;
  double* __restrict__ U = ws + h * w;
  const int hw = h * w;
  for (int base = tid; base < hw; base += kBatch * NT) {  // kBatch loads in flight
    double v[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) v[u] = base + u * NT < hw ? __ldcg(Lt + base + u * NT) : 0.0;
#pragma unroll
    for (int u = 0; u < kBatch; ++u)
      if (base + u * NT < hw) P[base + u * NT] = v[u];
  }
  for (int idx = tid; idx < m * m; idx += NT) U[idx] = 0.0;
  group_sync<NT>();
  extend_add<NT>(d, t, tid, P, h, w, U, srel);
  factor_panel<NT>(P, h, w, f, tid, tol, d.bad, d.Dinv);
  form_update<NT>(P, h, w, tid, U);
  group_sync<NT>();
  for (int idx = tid; idx < h * w; idx += NT) __stcg(Lt + idx, P[idx]);
  for (int idx = tid; idx < m * m; idx += NT) __stcg(Ut + idx, U[idx]);
}

// A group: its levels one after the other, a warp per supernode.
__device__ void group_factor(const CholDev& d, int g, double tol, double* smem, int* srel) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lp = __ldg(d.grp_lptr + g), nlv = __ldg(d.grp_lptr + g + 1) - lp - 1;
  double* ws = smem + warp * kSmallStage;
  int* wr = srel + warp * kCholWarpRows;
  for (int v = 0; v < nlv; ++v) {
    const int a = __ldg(d.grp_lev + lp + v), b = __ldg(d.grp_lev + lp + v + 1);
    for (int q = a + warp; q < b; q += kWarps) factor_staged<32>(d, __ldg(d.grp_sn + q), lane, tol, ws, wr);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// tiles of a large supernode's front
// ---------------------------------------------------------------------------
struct Front {
  double* L;  // panel, h x w, leading dimension h
  double* U;  // update matrix, m x m, leading dimension m
  int f, w, h, m, nbp;
  __device__ Front(const CholDev& d, int s) {
    f = __ldg(d.sn_first + s);
    w = __ldg(d.sn_first + s + 1) - f;
    h = __ldg(d.sn_rowptr + s + 1) - __ldg(d.sn_rowptr + s);
    m = h - w;
    nbp = (w + T - 1) / T;
    L = d.Lx + __ldg(d.sn_off + s);
    U = d.Ux + __ldg(d.u_off + s);
  }
  // first front row of tile row I and its row count (tiles do not straddle w)
  __device__ void span(int I, int& r0, int& len) const {
    if (I < nbp) {
      r0 = I * T;
      len = min(T, w - r0);
    } else {
      r0 = w + (I - nbp) * T;
      len = min(T, h - r0);
    }
  }
  // element (front row r, front column c), r >= c
  __device__ double* at(int r, int c) const {
    return c < w ? L + size_t(c) * h + r : U + size_t(c - w) * m + (r - w);
  }
  __device__ int ld(int c) const { return c < w ? h : m; }
};

// tile (rows r0.., cols c0..; nr x nc) of the front -> shared S (column-major,
// leading dimension T): a row per lane, T / kWarps columns per warp, all
// loads in flight together
constexpr int kColsPerWarp = T / kWarps;
__device__ __forceinline__ void tile_load(const Front& F, int r0, int nr, int c0, int nc,
                                          double* __restrict__ S) {
  const int lane = threadIdx.x & 31, w0 = threadIdx.x >> 5;
  if (lane < nr) {
    const double* src = F.at(r0 + lane, c0);
    const size_t ld = F.ld(c0);
    double v[kColsPerWarp];
#pragma unroll
    for (int u = 0; u < kColsPerWarp; ++u) {
      const int c = w0 + u * kWarps;
      v[u] = c < nc ? __ldcg(src + c * ld) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kColsPerWarp; ++u) S[(w0 + u * kWarps) * T + lane] = v[u];
  }
}
__device__ __forceinline__ void tile_store(const Front& F, int r0, int nr, int c0, int nc,
                                           const double* __restrict__ S) {
  const int lane = threadIdx.x & 31, w0 = threadIdx.x >> 5;
  if (lane < nr) {
    double* dst = F.at(r0 + lane, c0);
    const size_t ld = F.ld(c0);
#pragma unroll
    for (int u = 0; u < kColsPerWarp; ++u) {
      const int c = w0 + u * kWarps;
      if (c < nc) __stcg(dst + c * ld, S[c * T + lane]);
    }
  }
}

// Extend-add into tile (I, J): each child's update-matrix entries that land
// in the tile, child after child.  The children's row maps ascend, so the
// entries form one rectangle of the child's matrix: its rows [brk[I],
// brk[I + 1]) and columns [brk[J], brk[J + 1]), brk being the child's row
// positions at the parent's tile boundaries (computed on the host).
__device__ void tile_asm(const CholDev& d, int s, int I, int J, double* smem) {
  const Front F(d, s);
  int r0, nr, c0, nc;
  F.span(I, r0, nr);
  F.span(J, c0, nc);
  double* S = smem;
  tile_load(F, r0, nr, c0, nc, S);
  // children's descriptors and tile breakpoints, read one child ahead
  const int q0 = __ldg(d.kid_ptr + s), q1 = __ldg(d.kid_ptr + s + 1);
  int4 next = q0 < q1 ? __ldg(d.kid_desc + q0) : make_int4(0, 0, 0, 0);
  int next_brk = q0 < q1 ? __ldg(d.kid_brk + q0) : 0;
  for (int q = q0; q < q1; ++q) {
    const int4 kd = next;
    const int32_t* brk = d.tile_brk + next_brk;
    if (q + 1 < q1) {
      next = __ldg(d.kid_desc + q + 1);
      next_brk = __ldg(d.kid_brk + q + 1);
    }
    const int mc = kd.x;
    const int32_t* rel = d.relmap + kd.y;
    const int ia = __ldg(brk + I), ni = __ldg(brk + I + 1) - ia;
    const int ja = __ldg(brk + J), nj = __ldg(brk + J + 1) - ja;
    const double* __restrict__ Uc =
        d.Ux + ((static_cast<int64_t>(kd.w) << 32) | static_cast<uint32_t>(kd.z));
    __syncthreads();  // the tile is loaded / the previous child's additions are done
    for (int idx = threadIdx.x; idx < ni * nj; idx += kThreads) {
      const int i = ia + idx % ni, j = ja + idx / ni;
      if (i >= j) S[(__ldg(rel + j) - c0) * T + (__ldg(rel + i) - r0)] += __ldcg(Uc + size_t(j) * mc + i);
    }
  }
  __syncthreads();
  tile_store(F, r0, nr, c0, nc, S);
}

// Tile (I, k) <- tile (I, k) L_kk^-T by four warps (one per sub-partition):
// a row of the tile per lane, column j held by warp j mod 4 in registers.
// Step c: every warp subtracts the solved column c's multiple from its later
// columns; the owner of column c + 1 updates that column first, solves it
// (times 1 / L_kk[c+1][c+1]) into the ring buffer c + 1 mod 4 and announces
// it with a non-waiting arrival, the others wait for it (named barriers as
// in tile_potrf below).
constexpr int kTrsmWarps = 4;
constexpr int kTrsmCols = T / kTrsmWarps;
__device__ __forceinline__ void named_sync(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(32 * kTrsmWarps) : "memory");
}
__device__ __forceinline__ void named_arrive(int id) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "n"(32 * kTrsmWarps) : "memory");
}
__device__ void tile_trsm(const CholDev& d, int s, int I, int k, double* smem) {
  if (threadIdx.x >= 32 * kTrsmWarps) return;
  const Front F(d, s);
  int rk, n, r0, nr;
  F.span(k, rk, n);
  F.span(I, r0, nr);
  double* Ls = smem;               // L_kk, column-major
  double* rinv = smem + T * T;     // 1 / L_kk[c][c]
  double* Xs = smem + T * T + T;   // the solved columns, a ring of four
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  {  // L_kk: a row per lane, the warp's columns
    const double* src = F.at(rk + lane, rk);
    const size_t ld = F.ld(rk);
#pragma unroll
    for (int u = 0; u < kTrsmCols; ++u) {
      const int c = wp + kTrsmWarps * u;
      Ls[c * T + lane] = lane < n && c < n && c <= lane ? __ldcg(src + c * ld) : 0.0;
    }
  }
  double b[kTrsmCols];
  const double* src = F.at(r0 + (lane < nr ? lane : 0), rk);
  const size_t ldb = F.ld(rk);
#pragma unroll
  for (int u = 0; u < kTrsmCols; ++u) {
    const int c = wp + kTrsmWarps * u;
    b[u] = lane < nr && c < n ? __ldcg(src + c * ldb) : 0.0;
  }
  named_sync(1);
  if (wp == 0 && lane < n) rinv[lane] = 1.0 / Ls[lane * T + lane];
  named_sync(1);
  if (wp == 0) {  // column 0 needs no update
    b[0] *= rinv[0];
    Xs[lane] = b[0];
  }
  named_sync(2);
#pragma unroll
  for (int c = 0; c < T; ++c) {
    if (c < n) {
      const double* X = Xs + (c & 3) * T;
      const double xc = X[lane];
      const bool producer = c + 1 < n && wp == (c + 1) % kTrsmWarps;
      if (producer) {
        const int u1 = (c + 1) / kTrsmWarps;  // (a constant: c is unrolled)
#pragma unroll
        for (int u = 0; u < kTrsmCols; ++u)
          if (u == u1) {
            b[u] = fma(-xc, Ls[c * T + c + 1], b[u]) * rinv[c + 1];
            Xs[((c + 1) & 3) * T + lane] = b[u];
          }
        named_arrive(1 + (c & 1));
      }
#pragma unroll
      for (int u = 0; u < kTrsmCols; ++u) {
        const int j = wp + kTrsmWarps * u;
        if (j > c + 1 && j < n) b[u] = fma(-xc, Ls[c * T + j], b[u]);
      }
      if (!producer) named_sync(1 + (c & 1));
    }
  }
  if (lane < nr) {
    double* dst = F.at(r0 + lane, rk);
#pragma unroll
    for (int u = 0; u < kTrsmCols; ++u) {
      const int c = wp + kTrsmWarps * u;
      if (c < n) __stcg(dst + c * ldb, b[u]);
    }
  }
}

// Cholesky of diagonal tile k of the panel by four warps (one per
// sub-partition; pivot test as in factor_panel): a row of the tile per
// lane, column j held by warp j mod 4 in registers.  Step c: every warp
// subtracts column c's multiple from its later columns.  The owner of column
// c + 1 updates that column first, takes its pivot (reciprocal square root,
// scaled column into the ring buffer c + 1 mod 4) and announces it with a
// non-waiting arrival; the others wait for it at the step's barrier (named
// barriers 1 and 2 alternate, so a warp that arrives early cannot be counted
// in the previous step's barrier).  The chain of dependent work per column
// is one update, one reciprocal square root and one barrier.
__device__ void tile_potrf(const CholDev& d, int s, int k, double tol, double* smem) {
  if (threadIdx.x >= 32 * kTrsmWarps) return;
  const Front F(d, s);
  int r0, n;
  F.span(k, r0, n);
  double* Xs = smem;  // the scaled columns, a ring of four
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const size_t ld = F.ld(r0);
  double a[kTrsmCols];
  {
    const double* src = F.at(r0 + (lane < n ? lane : 0), r0);
#pragma unroll
    for (int u = 0; u < kTrsmCols; ++u) {
      const int c = wp + kTrsmWarps * u;
      a[u] = lane < n && c < n && c <= lane ? __ldcg(src + c * ld) : 0.0;
    }
  }
  // column c's pivot by its owner (register a[u]): L[c][c] and L[i][c]
  // (i > c) into a[u] and ring buffer c & 3
  auto pivot = [&](int c, int u) {
    double p = __shfl_sync(0xffffffffu, a[u], c);
    if (!(p > tol)) {
      if (lane == 0) atomicMin(d.bad, F.f + r0 + c);
      p = 1.0;
    }
    const double rinv = rsqrt(p);
    const double x = lane == c ? p * rinv : (lane > c ? a[u] * rinv : 0.0);
    a[u] = x;
    Xs[(c & 3) * T + lane] = x;
    if (lane == 0) d.Dinv[F.f + r0 + c] = rinv;
  };
  if (wp == 0 && n > 0) pivot(0, 0);
  named_sync(2);
#pragma unroll
  for (int c = 0; c < T; ++c) {
    if (c < n) {
      const double* X = Xs + (c & 3) * T;
      const double xi = X[lane];
      const bool producer = c + 1 < n && wp == (c + 1) % kTrsmWarps;
      if (producer) {  // the next column, its pivot, the announcement
        const int u1 = (c + 1) / kTrsmWarps;  // (a constant: c is unrolled)
#pragma unroll
        for (int u = 0; u < kTrsmCols; ++u)
          if (u == u1) {
            a[u] = fma(-xi, X[c + 1], a[u]);
            pivot(c + 1, u);
          }
        named_arrive(1 + (c & 1));
      }
#pragma unroll
      for (int u = 0; u < kTrsmCols; ++u) {
        const int j = wp + kTrsmWarps * u;
        if (j > c + 1 && j < n) a[u] = fma(-xi, X[j], a[u]);
      }
      if (!producer) named_sync(1 + (c & 1));
    }
  }
  if (lane < n) {
    double* dst = F.at(r0 + lane, r0);
#pragma unroll
    for (int u = 0; u < kTrsmCols; ++u) {
      const int c = wp + kTrsmWarps * u;
      if (c < n && c <= lane) __stcg(dst + c * ld, a[u]);
    }
  }
}

// Tile (I, J) -= tile (I, k) tile (J, k)' (lower part of a diagonal tile).
// Off the diagonal: rows over the lanes, a column per warp and round.  On
// it: the lower triangle's entries (column by column) spread evenly over
// all threads, so that no warp issues FMAs for the upper triangle (an FP64
// warp instruction costs the same however few lanes are active; the
// diagonal updates lie on the factorization's critical path).
__device__ void tile_upd(const CholDev& d, int s, int I, int J, int k, double* smem) {
  const Front F(d, s);
  int rk, n, r0, nr, c0, nc;
  F.span(k, rk, n);
  F.span(I, r0, nr);
  F.span(J, c0, nc);
  double* As = smem;
  double* Bs = smem + T * T;
  tile_load(F, r0, nr, rk, n, As);
  tile_load(F, c0, nc, rk, n, Bs);
  __syncthreads();
  const int ld = F.ld(c0);
  if (I == J) {  // nr == nc
    const int ne = nr * (nr + 1) / 2;
    for (int e = threadIdx.x; e < ne; e += kThreads) {
      int j = 0, st = 0;  // column j's entries start at st
      while (st + (nr - j) <= e) {
        st += nr - j;
        ++j;
      }
      const int i = j + (e - st);
      double acc = 0.0;
      for (int q = 0; q < n; ++q) acc = fma(As[q * T + i], Bs[q * T + j], acc);
      double* C = F.at(r0 + i, c0) + size_t(j) * ld;
      __stcg(C, __ldcg(C) - acc);
    }
    return;
  }
  const int i = int(threadIdx.x & 31);
  if (i >= nr) return;
  double* C = F.at(r0 + i, c0);
  for (int j = int(threadIdx.x >> 5); j < nc; j += kWarps) {
    double acc = 0.0;
    for (int q = 0; q < n; ++q) acc = fma(As[q * T + i], Bs[q * T + j], acc);
    __stcg(C + size_t(j) * ld, __ldcg(C + size_t(j) * ld) - acc);
  }
}

// ---------------------------------------------------------------------------
// bottom levels: one thread per supernode (at most kCholBottomRows rows,
// kCholBottomCols columns), its panel and the lower triangle of its update
// matrix staged in shared memory, element e of thread t at [e * kBotThreads
// + t] (so a warp's accesses fall on distinct banks)
// ---------------------------------------------------------------------------
constexpr int kBotThreads = 64;
constexpr int kBotBatch = 16;   // global loads a thread keeps in flight
// per-thread staging: the child's row map (kCholBottomRows ints, as doubles'
// worth of space) then the panel and the packed lower update matrix
constexpr int kBotMap = kCholBottomRows / 2;
static_assert(kCholBottomRows == 16 && kCholBottomCols == 4, "staging is sized for 16 x 4");

// `stage`: doubles of staging per thread for this level (at most kBotMap +
// 142: h w + m (m + 1) / 2 <= 142 for h <= 16, w <= 4).
__global__ void __launch_bounds__(kBotThreads) k_chol_bottom(CholDev d, const int32_t* __restrict__ list,
                                                              int count, double tol) {
  extern __shared__ double sb[];
  const int q = blockIdx.x * kBotThreads + threadIdx.x;
  if (q >= count) return;
  int* __restrict__ R = reinterpret_cast<int*>(sb) + threadIdx.x;  // R[i * kBotThreads]
  double* __restrict__ S = sb + kBotMap * kBotThreads + threadIdx.x;
  const int s = __ldg(list + q);
  const int f = __ldg(d.sn_first + s), w = __ldg(d.sn_first + s + 1) - f;
  const int h = __ldg(d.sn_rowptr + s + 1) - __ldg(d.sn_rowptr + s), m = h - w, hw = h * w;
  double* __restrict__ Lt = d.Lx + __ldg(d.sn_off + s);
  double* __restrict__ Ut = d.Ux + __ldg(d.u_off + s);
  // packed lower update matrix: column j at hw + j m - j (j - 1) / 2
  auto uix = [&](int i, int j) { return hw + j * m - (j * (j - 1)) / 2 + (i - j); };
  // the panel, kBotBatch loads in flight at a time
  for (int e0 = 0; e0 < hw; e0 += kBotBatch) {
    double v[kBotBatch];
#pragma unroll
    for (int u = 0; u < kBotBatch; ++u) v[u] = e0 + u < hw ? Lt[e0 + u] : 0.0;
#pragma unroll
    for (int u = 0; u < kBotBatch; ++u)
      if (e0 + u < hw) S[(e0 + u) * kBotThreads] = v[u];
  }
  for (int e = hw; e < hw + m * (m + 1) / 2; ++e) S[e * kBotThreads] = 0.0;
  for (int k = __ldg(d.kid_ptr + s); k < __ldg(d.kid_ptr + s + 1); ++k) {
    const int c = __ldg(d.kid + k);
    const int mc = (__ldg(d.sn_rowptr + c + 1) - __ldg(d.sn_rowptr + c)) -
                   (__ldg(d.sn_first + c + 1) - __ldg(d.sn_first + c));
    const double* __restrict__ Uc = d.Ux + __ldg(d.u_off + c);
    const int32_t* __restrict__ rel = d.relmap + __ldg(d.rel_off + c);
    {  // the child's row map (at most kCholBottomRows - 1 rows below its columns)
      int rv[kCholBottomRows];
#pragma unroll
      for (int u = 0; u < kCholBottomRows; ++u) rv[u] = u < mc ? __ldg(rel + u) : 0;
#pragma unroll
      for (int u = 0; u < kCholBottomRows; ++u) R[u * kBotThreads] = rv[u];
    }
    // its lower triangle, column by column, kBotBatch entries in flight at a time
    int i = 0, j = 0;
    const int nl = mc * (mc + 1) / 2;
    for (int e0 = 0; e0 < nl; e0 += kBotBatch) {
      double v[kBotBatch];
      int ij[kBotBatch];
#pragma unroll
      for (int u = 0; u < kBotBatch; ++u) {
        ij[u] = (j << 8) | i;
        v[u] = e0 + u < nl ? Uc[size_t(j) * mc + i] : 0.0;
        if (++i == mc) {
          ++j;
          i = j;
        }
      }
#pragma unroll
      for (int u = 0; u < kBotBatch; ++u) {
        if (e0 + u >= nl) continue;
        const int ri = R[(ij[u] & 0xff) * kBotThreads], rj = R[(ij[u] >> 8) * kBotThreads];
        const int e = rj < w ? rj * h + ri : uix(ri - w, rj - w);
        S[e * kBotThreads] += v[u];
      }
    }
  }
  for (int k = 0; k < w; ++k) {
    double p = S[(k * h + k) * kBotThreads];
    if (!(p > tol)) {
      atomicMin(d.bad, f + k);
      p = 1.0;
    }
    const double rinv = rsqrt(p), r = p * rinv;
    S[(k * h + k) * kBotThreads] = r;
    d.Dinv[f + k] = rinv;
    for (int i = k + 1; i < h; ++i) S[(k * h + i) * kBotThreads] *= rinv;
    for (int j = k + 1; j < w; ++j) {
      const double ljk = S[(k * h + j) * kBotThreads];
      for (int i = j; i < h; ++i) S[(j * h + i) * kBotThreads] -= S[(k * h + i) * kBotThreads] * ljk;
    }
  }
  for (int j = 0; j < m; ++j)
    for (int i = j; i < m; ++i) {
      double acc = 0.0;
      for (int k = 0; k < w; ++k)
        acc = fma(S[(k * h + w + i) * kBotThreads], S[(k * h + w + j) * kBotThreads], acc);
      S[uix(i, j) * kBotThreads] -= acc;
    }
  for (int e = 0; e < hw; ++e) Lt[e] = S[e * kBotThreads];
  for (int j = 0; j < m; ++j)
    for (int i = j; i < m; ++i) Ut[size_t(j) * m + i] = S[uix(i, j) * kBotThreads];
}

// Forward substitution of the bottom supernodes of one level, a thread each.
__global__ void __launch_bounds__(kThreads) k_chol_bottom_fwd(CholDev d, const int32_t* __restrict__ list,
                                                               int count, double* __restrict__ y) {
  const int q = blockIdx.x * kThreads + threadIdx.x;
  if (q >= count) return;
  const int s = __ldg(list + q);
  const int f = __ldg(d.sn_first + s), w = __ldg(d.sn_first + s + 1) - f;
  const int h = __ldg(d.sn_rowptr + s + 1) - __ldg(d.sn_rowptr + s), m = h - w;
  const double* __restrict__ Lt = d.Lx + __ldg(d.sn_off + s);
  double* __restrict__ zt = d.Zx + __ldg(d.z_off + s);
  for (int k = __ldg(d.kid_ptr + s); k < __ldg(d.kid_ptr + s + 1); ++k) {
    const int c = __ldg(d.kid + k);
    const int mc = (__ldg(d.sn_rowptr + c + 1) - __ldg(d.sn_rowptr + c)) -
                   (__ldg(d.sn_first + c + 1) - __ldg(d.sn_first + c));
    const double* __restrict__ zc = d.Zx + __ldg(d.z_off + c);
    const int32_t* __restrict__ rel = d.relmap + __ldg(d.rel_off + c);
    double v[kCholBottomRows];
    int r[kCholBottomRows];
#pragma unroll
    for (int i = 0; i < kCholBottomRows; ++i) {
      v[i] = i < mc ? zc[i] : 0.0;
      r[i] = i < mc ? __ldg(rel + i) : 0;
    }
#pragma unroll
    for (int i = 0; i < kCholBottomRows; ++i) {
      if (i >= mc) continue;
      if (r[i] < w)
        y[f + r[i]] += v[i];
      else
        zt[r[i] - w] += v[i];
    }
  }
  double yv[kCholBottomCols];
  for (int k = 0; k < w; ++k) {
    const double yk = y[f + k] * d.Dinv[f + k];
    y[f + k] = yk;
    for (int i = k + 1; i < w; ++i) y[f + i] -= Lt[size_t(k) * h + i] * yk;
  }
#pragma unroll
  for (int k = 0; k < kCholBottomCols; ++k) yv[k] = k < w ? y[f + k] : 0.0;
  for (int i = 0; i < m; ++i) {
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < kCholBottomCols; ++k)
      if (k < w) acc = fma(Lt[size_t(k) * h + w + i], yv[k], acc);
    zt[i] -= acc;
  }
}

// Backward substitution of the bottom supernodes of one level, a thread each.
__global__ void __launch_bounds__(kThreads) k_chol_bottom_bwd(CholDev d, const int32_t* __restrict__ list,
                                                               int count, double* __restrict__ x) {
  const int q = blockIdx.x * kThreads + threadIdx.x;
  if (q >= count) return;
  const int s = __ldg(list + q);
  const int f = __ldg(d.sn_first + s), w = __ldg(d.sn_first + s + 1) - f;
  const int r0 = __ldg(d.sn_rowptr + s), h = __ldg(d.sn_rowptr + s + 1) - r0;
  const double* __restrict__ Lt = d.Lx + __ldg(d.sn_off + s);
  double xb[kCholBottomRows];  // x at the rows below the supernode's columns
#pragma unroll
  for (int i = 0; i < kCholBottomRows; ++i) xb[i] = w + i < h ? x[__ldg(d.rowidx + r0 + w + i)] : 0.0;
  for (int k = 0; k < w; ++k) {
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < kCholBottomRows; ++i)
      if (w + i < h) acc = fma(Lt[size_t(k) * h + w + i], xb[i], acc);
    x[f + k] -= acc;
  }
  for (int k = w - 1; k >= 0; --k) {
    const double xk = x[f + k] * d.Dinv[f + k];
    x[f + k] = xk;
    for (int i = 0; i < k; ++i) x[f + i] -= Lt[size_t(i) * h + k] * xk;
  }
}

__global__ void __launch_bounds__(kThreads, 2) k_chol_factor_tasks(CholDev d, CholTasks g,
                                                                    double tol) {
  extern __shared__ double smem[];
  int* srel = reinterpret_cast<int*>(smem + kStageDoubles);
  task_loop(g, d.abort, [](int4) { return 0; }, [&](int4 tk, int) {
    const int kind = tk.x & 0xff, k = tk.x >> 8;
    switch (kind) {
      case kTaskGroup: group_factor(d, tk.y, tol, smem, srel); break;
      case kTaskBlock: factor_staged<kThreads>(d, tk.y, threadIdx.x, tol, smem, srel); break;
      case kTaskAsm: tile_asm(d, tk.y, tk.z, tk.w, smem); break;
      case kTaskPotrf: tile_potrf(d, tk.y, k, tol, smem); break;
      case kTaskTrsm: tile_trsm(d, tk.y, tk.z, k, smem); break;
      case kTaskUpd: tile_upd(d, tk.y, tk.z, tk.w, k, smem); break;
      default: break;  // fin: no work
    }
  });
  wait_prior_grid();
}

// ---------------------------------------------------------------------------
// solves
// ---------------------------------------------------------------------------
// The children's update vectors of t: entries in t's columns go to y, the
// rest to t's update vector zt.
template <int NT>
__device__ void add_children_z(const CholDev& d, int t, int tid, int f, int w,
                               double* __restrict__ y, double* __restrict__ zt) {
  for (int q = __ldg(d.kid_ptr + t); q < __ldg(d.kid_ptr + t + 1); ++q) {
    const int c = __ldg(d.kid + q);
    const int mc = (__ldg(d.sn_rowptr + c + 1) - __ldg(d.sn_rowptr + c)) -
                   (__ldg(d.sn_first + c + 1) - __ldg(d.sn_first + c));
    const double* __restrict__ zc = d.Zx + __ldg(d.z_off + c);
    const int32_t* __restrict__ rel = d.relmap + __ldg(d.rel_off + c);
    for (int ii = tid; ii < mc; ii += NT) {
      const int r = __ldg(rel + ii);
      double* dst = r < w ? y + f + r : zt + (r - w);
      __stcg(dst, __ldcg(dst) + __ldcg(zc + ii));
    }
    group_sync<NT>();
  }
}

// Gather-list entries a row of a solve task keeps in registers from before
// its dependencies are done (longer lists load the rest afterwards).
constexpr int kGatherRegs = 4;

// Forward substitution of one supernode by one warp (small supernodes), in
// two parts.  Before the wait (forward_small_pre): everything no dependency
// writes: the panel (the factorization's, a kernel before), staged in the
// warp's slice `ws`; y at the supernode's own columns (no other task writes
// it); the pivots' reciprocals; each row's gather list.  After it
// (forward_small_run): the children's update-vector entries, summed per row
// in child order onto y_t (rows below: onto zero); the diagonal block (y_t
// in the lanes, row r in lane r); z_t = (gathered) - L21 y_t; each stored
// once.
struct FwdSmall {
  int f, w, h, p0, cnt;
  double* zt;
  double y0, di;
  int idx[kGatherRegs];
};

__device__ FwdSmall forward_small_pre(const CholDev& d, int t, int lane,
                                      const double* __restrict__ y, double* __restrict__ ws) {
  FwdSmall s;
  s.f = __ldg(d.sn_first + t);
  s.w = __ldg(d.sn_first + t + 1) - s.f;
  const int r0 = __ldg(d.sn_rowptr + t);
  s.h = __ldg(d.sn_rowptr + t + 1) - r0;
  const double* __restrict__ Lt = d.Lx + __ldg(d.sn_off + t);
  s.zt = d.Zx + __ldg(d.z_off + t);
  double v[kSmallPanel / 32];
#pragma unroll
  for (int u = 0; u < kSmallPanel / 32; ++u) {
    const int e = lane + 32 * u;
    v[u] = e < s.h * s.w ? __ldcg(Lt + e) : 0.0;
  }
  s.y0 = lane < s.w ? __ldcg(y + s.f + lane) : 0.0;
  s.di = lane < s.w ? __ldcg(d.Dinv + s.f + lane) : 0.0;
  s.p0 = lane < s.h ? __ldg(d.fg_ptr + r0 + lane) : 0;
  s.cnt = lane < s.h ? __ldg(d.fg_ptr + r0 + lane + 1) - s.p0 : 0;
#pragma unroll
  for (int u = 0; u < kSmallPanel / 32; ++u) ws[lane + 32 * u] = v[u];
#pragma unroll
  for (int u = 0; u < kGatherRegs; ++u) s.idx[u] = u < s.cnt ? __ldg(d.fg_idx + s.p0 + u) : 0;
  __syncwarp();
  return s;
}

__device__ void forward_small_run(const CholDev& d, const FwdSmall& s, int lane,
                                  double* __restrict__ y, const double* __restrict__ ws) {
  double zv[kGatherRegs];
#pragma unroll
  for (int u = 0; u < kGatherRegs; ++u) zv[u] = u < s.cnt ? __ldcg(d.Zx + s.idx[u]) : 0.0;
  double acc = s.y0;  // rows >= w: 0
#pragma unroll
  for (int u = 0; u < kGatherRegs; ++u)
    if (u < s.cnt) acc += zv[u];
  for (int q = kGatherRegs; q < s.cnt; ++q) acc += __ldcg(d.Zx + __ldg(d.fg_idx + s.p0 + q));
  const int w = s.w, h = s.h, m = h - w;
  double yv = lane < w ? acc : 0.0;
  for (int k = 0; k < w; ++k) {
    const double yk = __shfl_sync(0xffffffffu, yv * s.di, k);
    if (lane == k) yv = yk;
    if (lane > k && lane < w) yv = fma(-ws[k * h + lane], yk, yv);
  }
  if (lane < w) __stcg(y + s.f + lane, yv);
  double z = __shfl_sync(0xffffffffu, acc, (w + lane) & 31);  // row w + lane
  if (lane >= m) z = 0.0;
  for (int k = 0; k < w; ++k) {
    const double yk = __shfl_sync(0xffffffffu, yv, k);
    if (lane < m) z = fma(-ws[k * h + w + lane], yk, z);
  }
  if (lane < m) __stcg(s.zt + lane, z);
  __syncwarp();  // the slice is reused by the warp's next supernode
}

// The same by a whole block for a supernode whose update vector exceeds the
// staged solves' capacity (below): the diagonal block and y_t staged in
// shared memory, the triangular solve done by the first warp, the update
// vector accumulated in global memory.
__device__ void forward_large(const CholDev& d, int t, double* __restrict__ y,
                              double* __restrict__ sL, double* __restrict__ sy) {
  const int f = __ldg(d.sn_first + t), w = __ldg(d.sn_first + t + 1) - f;
  const int h = __ldg(d.sn_rowptr + t + 1) - __ldg(d.sn_rowptr + t), m = h - w;
  const double* __restrict__ Lt = d.Lx + __ldg(d.sn_off + t);
  double* __restrict__ zt = d.Zx + __ldg(d.z_off + t);
  add_children_z<kThreads>(d, t, threadIdx.x, f, w, y, zt);
  for (int idx = threadIdx.x; idx < w * w; idx += kThreads) {
    const int k = idx / w, i = idx - k * w;
    sL[idx] = __ldcg(Lt + size_t(k) * h + i);
  }
  for (int k = threadIdx.x; k < w; k += kThreads) sy[k] = __ldcg(y + f + k);
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int k = 0; k < w; ++k) {
      const double yk = sy[k] * __ldcg(d.Dinv + f + k);
      __syncwarp();
      if (lane == 0) sy[k] = yk;
      for (int i = k + 1 + lane; i < w; i += 32) sy[i] -= sL[k * w + i] * yk;
      __syncwarp();
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < w; k += kThreads) __stcg(y + f + k, sy[k]);
  for (int i = threadIdx.x; i < m; i += kThreads) {
    double acc = 0.0;
    for (int k = 0; k < w; ++k) acc = fma(__ldcg(Lt + size_t(k) * h + w + i), sy[k], acc);
    __stcg(zt + i, __ldcg(zt + i) - acc);
  }
}

// Backward substitution of one supernode by one warp (small supernodes):
// x_t -= L21' x(R_t below) (fixed reduction trees), then the transposed
// diagonal block (x_t in the lanes).  Before the wait: the panel (staged
// in `ws`), x_t (the forward solve's result: no backward task but this one
// writes it), the pivots' reciprocals and the rows below; after it: x at
// those rows (the ancestors' results).
struct BwdSmall {
  int f, w, h, ri;
  double xv, di;
};

__device__ BwdSmall backward_small_pre(const CholDev& d, int t, int lane,
                                       const double* __restrict__ x, double* __restrict__ ws) {
  BwdSmall s;
  s.f = __ldg(d.sn_first + t);
  s.w = __ldg(d.sn_first + t + 1) - s.f;
  const int r0 = __ldg(d.sn_rowptr + t);
  s.h = __ldg(d.sn_rowptr + t + 1) - r0;
  const int m = s.h - s.w;
  const double* __restrict__ Lt = d.Lx + __ldg(d.sn_off + t);
  s.ri = lane < m ? __ldg(d.rowidx + r0 + s.w + lane) : 0;
  s.xv = lane < s.w ? __ldcg(x + s.f + lane) : 0.0;
  s.di = lane < s.w ? __ldcg(d.Dinv + s.f + lane) : 0.0;
  double v[kSmallPanel / 32];
#pragma unroll
  for (int u = 0; u < kSmallPanel / 32; ++u) {
    const int e = lane + 32 * u;
    v[u] = e < s.h * s.w ? __ldcg(Lt + e) : 0.0;
  }
#pragma unroll
  for (int u = 0; u < kSmallPanel / 32; ++u) ws[lane + 32 * u] = v[u];
  __syncwarp();
  return s;
}

__device__ void backward_small_run(const BwdSmall& s, int lane, double* __restrict__ x,
                                   const double* __restrict__ ws) {
  const int w = s.w, h = s.h, m = h - w;
  const double xb = lane < m ? __ldcg(x + s.ri) : 0.0;
  double xv = s.xv;
  {
    // x_t[k] -= sum_i L21[i][k] x_b[i]: lane = g wp + k (wp = w rounded up
    // to a power of two, G = 32 / wp row groups) sums rows g, g + G, ... in
    // order, then the G partial sums of column k meet in a fixed tree: few
    // FP64 instructions per column, which bound the warp-task phase
    const int wp = w <= 1 ? 1 : (w <= 2 ? 2 : (w <= 4 ? 4 : 8)), G = 32 / wp;
    const int k = lane & (wp - 1), g = lane / wp;
    double acc = 0.0;
    for (int i = g; i - g < m; i += G) {
      const double xi = __shfl_sync(0xffffffffu, xb, i & 31);
      if (k < w && i < m) acc = fma(ws[k * h + w + i], xi, acc);
    }
    for (int o = wp; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane < w) xv -= acc;
  }
  for (int k = w - 1; k >= 0; --k) {
    const double xk = __shfl_sync(0xffffffffu, xv * s.di, k);
    if (lane == k) xv = xk;
    if (lane < k) xv = fma(-ws[lane * h + k], xk, xv);
  }
  if (lane < w) __stcg(x + s.f + lane, xv);
  __syncwarp();
}

__device__ void backward_large(const CholDev& d, int t, double* __restrict__ x,
                               double* __restrict__ sL, double* __restrict__ sx) {
  const int f = __ldg(d.sn_first + t), w = __ldg(d.sn_first + t + 1) - f;
  const int r0 = __ldg(d.sn_rowptr + t), h = __ldg(d.sn_rowptr + t + 1) - r0;
  const double* __restrict__ Lt = d.Lx + __ldg(d.sn_off + t);
  const int lane = threadIdx.x & 31;
  for (int k = threadIdx.x >> 5; k < w; k += kWarps) {
    double acc = 0.0;
    for (int i = w + lane; i < h; i += 32)
      acc = fma(__ldcg(Lt + size_t(k) * h + i), __ldcg(x + __ldg(d.rowidx + r0 + i)), acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) sx[k] = __ldcg(x + f + k) - acc;
  }
  for (int idx = threadIdx.x; idx < w * w; idx += kThreads) {
    const int k = idx / w, i = idx - k * w;
    sL[idx] = __ldcg(Lt + size_t(k) * h + i);
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    for (int k = w - 1; k >= 0; --k) {
      const double xk = sx[k] * __ldcg(d.Dinv + f + k);
      __syncwarp();
      if (lane == 0) sx[k] = xk;
      for (int i = lane; i < k; i += 32) sx[i] -= sL[i * w + k] * xk;
      __syncwarp();
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < w; k += kThreads) __stcg(x + f + k, sx[k]);
}

// Staged block-task solves: a supernode whose update vector fits
// kSolveZCap doubles keeps its whole front in shared memory (the diagonal
// block, its reciprocal pivots, y_t or x_t, the update vector or the
// gathered solution below), the diagonal block is solved by warp 0 in
// registers (rows lane and lane + 32) with shuffles, and every vector is
// read and written in global memory once.
constexpr int kSolveZCap = 1024;
struct SolveStage {
  double* L;    // w x w diagonal block, columns scaled by 1 / L[j][j] (stage_diag)
  double* v;    // w: y_t / x_t
  double* di;   // w: 1 / L[j][j]
  double* z;    // m <= kSolveZCap: update vector / gathered x below
};

// Global loads a thread of the staged solves keeps in flight.
constexpr int kSolveBatch = 16;

// The diagonal block with each column scaled by its pivot's reciprocal,
// L_tt diag(L_tt)^-1 (unit diagonal, the diagonal itself not stored): the
// substitutions then carry one FMA per step on their dependent chain, the
// pivots applied once to the whole vector (forward: after, backward:
// before).
__device__ void stage_diag(const CholDev& d, const double* __restrict__ Lt, int f, int w, int h,
                           const SolveStage& S) {
  for (int base = threadIdx.x; base < w * w; base += kSolveBatch * kThreads) {
    double v[kSolveBatch], dk[kSolveBatch];
#pragma unroll
    for (int u = 0; u < kSolveBatch; ++u) {
      const int idx = base + u * kThreads, k = idx / w, i = idx - k * w;
      const bool in = idx < w * w && i > k;
      v[u] = in ? __ldcg(Lt + size_t(k) * h + i) : 0.0;
      dk[u] = in ? __ldcg(d.Dinv + f + k) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kSolveBatch; ++u)
      if (base + u * kThreads < w * w) S.L[base + u * kThreads] = v[u] * dk[u];
  }
  for (int i = threadIdx.x; i < w; i += kThreads) S.di[i] = __ldcg(d.Dinv + f + i);
}

// Threads per row of the forward step's z_t = (gathered) - L21 y_t and per
// column of the backward step's x_t -= L21' x(below).
__device__ __forceinline__ int fwd_row_threads(int w) {
  return w <= kSolveBatch ? 1 : (w <= 2 * kSolveBatch ? 2 : 4);
}
__device__ __forceinline__ int bwd_col_threads(int w) {
  int P = 32;  // the most (a power of two) that fit
  while (P > 1 && w * P > kThreads) P >>= 1;
  return P;
}

// A staged step in two parts, like the warp tasks': before the wait, the
// diagonal block and pivots into shared memory, the supernode's own entries
// of y (forward) or x (backward), the thread's row's gather list (forward)
// or row index below (backward), and the thread's first batch of L21 in
// registers; after it, the entries the dependencies wrote, then the solve.
struct StagedPre {
  bool staged;
  int f, w, h, r0;
  int p0, cnt, ri;
  int idx[kGatherRegs];
  double lv[kSolveBatch];
};

__device__ bool staged_shape(const CholDev& d, int t, StagedPre& s) {
  s.f = __ldg(d.sn_first + t);
  s.w = __ldg(d.sn_first + t + 1) - s.f;
  s.r0 = __ldg(d.sn_rowptr + t);
  s.h = __ldg(d.sn_rowptr + t + 1) - s.r0;
  s.staged = s.h - s.w <= kSolveZCap;
  return s.staged;
}

__device__ StagedPre forward_staged_pre(const CholDev& d, int t, const double* __restrict__ y,
                                        const SolveStage& S) {
  StagedPre s;
  if (!staged_shape(d, t, s)) return s;
  const int f = s.f, w = s.w, h = s.h, m = h - w, tid = threadIdx.x;
  const double* __restrict__ Lt = d.Lx + __ldg(d.sn_off + t);
  s.p0 = tid < h ? __ldg(d.fg_ptr + s.r0 + tid) : 0;
  s.cnt = tid < h ? __ldg(d.fg_ptr + s.r0 + tid + 1) - s.p0 : 0;
  {
    const int P = fwd_row_threads(w), part = tid & (P - 1), i = tid / P;
#pragma unroll
    for (int u = 0; u < kSolveBatch; ++u) {
      const int k = part + P * u;
      s.lv[u] = i < m && k < w ? __ldcg(Lt + size_t(k) * h + w + i) : 0.0;
    }
  }
  stage_diag(d, Lt, f, w, h, S);
  for (int i = tid; i < w; i += kThreads) S.v[i] = __ldcg(y + f + i);
#pragma unroll
  for (int u = 0; u < kGatherRegs; ++u) s.idx[u] = u < s.cnt ? __ldg(d.fg_idx + s.p0 + u) : 0;
  return s;
}

__device__ void forward_staged_run(const CholDev& d, int t, double* __restrict__ y,
                                   const SolveStage& S, const StagedPre& s) {
  const int f = s.f, w = s.w, h = s.h, m = h - w, tid = threadIdx.x;
  const double* __restrict__ Lt = d.Lx + __ldg(d.sn_off + t);
  double* __restrict__ zt = d.Zx + __ldg(d.z_off + t);
  // the children's update vectors: each row sums its gather list in child
  // order onto y_t (rows below: onto zero)
  for (int r = tid; r < h; r += kThreads) {
    double acc = r < w ? S.v[r] : 0.0;
    if (r == tid) {
      double zv[kGatherRegs];
#pragma unroll
      for (int u = 0; u < kGatherRegs; ++u) zv[u] = u < s.cnt ? __ldcg(d.Zx + s.idx[u]) : 0.0;
#pragma unroll
      for (int u = 0; u < kGatherRegs; ++u)
        if (u < s.cnt) acc += zv[u];
      for (int q = kGatherRegs; q < s.cnt; ++q) acc += __ldcg(d.Zx + __ldg(d.fg_idx + s.p0 + q));
    } else {
      const int q1 = __ldg(d.fg_ptr + s.r0 + r + 1);
      for (int q = __ldg(d.fg_ptr + s.r0 + r); q < q1; ++q)
        acc += __ldcg(d.Zx + __ldg(d.fg_idx + q));
    }
    if (r < w)
      S.v[r] = acc;
    else
      S.z[r - w] = acc;
  }
  __syncthreads();
  if (tid < 32) {  // y_t <- L_tt^-1 y_t: u = (unit block)^-1 y_t, y_t = u / pivots
    const int lane = tid;
    double u0 = lane < w ? S.v[lane] : 0.0, u1 = lane + 32 < w ? S.v[lane + 32] : 0.0;
    for (int k = 0; k < w; ++k) {
      const double* Lk = S.L + k * w;
      if (k < 32) {
        const double uk = __shfl_sync(0xffffffffu, u0, k);
        if (lane > k && lane < w) u0 = fma(-Lk[lane], uk, u0);
        if (lane + 32 < w) u1 = fma(-Lk[lane + 32], uk, u1);
      } else {
        const double uk = __shfl_sync(0xffffffffu, u1, k - 32);
        if (lane + 32 > k && lane + 32 < w) u1 = fma(-Lk[lane + 32], uk, u1);
      }
    }
    if (lane < w) S.v[lane] = u0 * S.di[lane];
    if (lane + 32 < w) S.v[lane + 32] = u1 * S.di[lane + 32];
  }
  __syncthreads();
  for (int i = tid; i < w; i += kThreads) __stcg(y + f + i, S.v[i]);
  // z_t = (gathered) - L21 y_t: each row's dot product split over P threads,
  // a thread's kSolveBatch loads in flight together (the first batch loaded
  // before the wait)
  const int P = fwd_row_threads(w);
  const int part = tid & (P - 1);
  for (int i0 = 0; i0 < m; i0 += kThreads / P) {
    const int i = i0 + tid / P;
    double v[kSolveBatch];
    if (i0 == 0) {
#pragma unroll
      for (int u = 0; u < kSolveBatch; ++u) v[u] = s.lv[u];
    } else {
#pragma unroll
      for (int u = 0; u < kSolveBatch; ++u) {
        const int k = part + P * u;
        v[u] = i < m && k < w ? __ldcg(Lt + size_t(k) * h + w + i) : 0.0;
      }
    }
    double acc = 0.0;
#pragma unroll
    for (int u = 0; u < kSolveBatch; ++u) {
      if (P * u >= w) break;  // the same for the whole warp: no empty FP64 issues
      const int k = part + P * u;
      if (k < w) acc = fma(v[u], S.v[k], acc);
    }
    for (int o = P / 2; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, P);
    if (i < m && part == 0) __stcg(zt + i, S.z[i] - acc);
  }
}

__device__ StagedPre backward_staged_pre(const CholDev& d, int t, const double* __restrict__ x,
                                         const SolveStage& S) {
  StagedPre s;
  if (!staged_shape(d, t, s)) return s;
  const int f = s.f, w = s.w, h = s.h, m = h - w, tid = threadIdx.x;
  const double* __restrict__ Lt = d.Lx + __ldg(d.sn_off + t);
  s.ri = tid < m ? __ldg(d.rowidx + s.r0 + w + tid) : 0;
  {
    const int P = bwd_col_threads(w), part = tid & (P - 1), k = tid / P;
#pragma unroll
    for (int u = 0; u < kSolveBatch; ++u) {
      const int i = part + P * u;
      s.lv[u] = k < w && i < m ? __ldcg(Lt + size_t(k) * h + w + i) : 0.0;
    }
  }
  stage_diag(d, Lt, f, w, h, S);
  for (int i = tid; i < w; i += kThreads) S.v[i] = __ldcg(x + f + i);
  return s;
}

__device__ void backward_staged_run(const CholDev& d, int t, double* __restrict__ x,
                                    const SolveStage& S, const StagedPre& s) {
  const int f = s.f, w = s.w, h = s.h, m = h - w, tid = threadIdx.x, lane = tid & 31;
  const double* __restrict__ Lt = d.Lx + __ldg(d.sn_off + t);
  for (int i = tid; i < m; i += kThreads)
    S.z[i] = __ldcg(x + (i == tid ? s.ri : __ldg(d.rowidx + s.r0 + w + i)));
  __syncthreads();
  // x_t -= L21' x(below): column k's dot product by P threads per column
  {
    const int P = bwd_col_threads(w);
    const int part = tid & (P - 1);
    for (int k0 = 0; k0 < w; k0 += kThreads / P) {
      const int k = k0 + tid / P;
      double acc = 0.0;
      for (int b = 0; b < m; b += P * kSolveBatch) {  // kSolveBatch loads in flight
        double v[kSolveBatch];
        if (k0 == 0 && b == 0) {
#pragma unroll
          for (int u = 0; u < kSolveBatch; ++u) v[u] = s.lv[u];
        } else {
#pragma unroll
          for (int u = 0; u < kSolveBatch; ++u) {
            const int i = b + part + P * u;
            v[u] = k < w && i < m ? __ldcg(Lt + size_t(k) * h + w + i) : 0.0;
          }
        }
#pragma unroll
        for (int u = 0; u < kSolveBatch; ++u) {
          if (b + P * u >= m) break;  // the same for the whole warp
          const int i = b + part + P * u;
          if (i < m) acc = fma(v[u], S.z[i], acc);
        }
      }
      for (int o = P / 2; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, P);
      if (k < w && part == 0) S.v[k] -= acc;
    }
  }
  __syncthreads();
  if (tid < 32) {  // x_t <- L_tt^-T x_t: the pivots first, then the unit block's transpose
    double x0 = lane < w ? S.v[lane] * S.di[lane] : 0.0;
    double x1 = lane + 32 < w ? S.v[lane + 32] * S.di[lane + 32] : 0.0;
    for (int k = w - 1; k >= 0; --k) {
      // row k of the unit block below the diagonal, read by column: U[k][i] = S.L(i * w + k)
      if (k >= 32) {
        const double xk = __shfl_sync(0xffffffffu, x1, k - 32);
        if (lane + 32 < k) x1 = fma(-S.L[(lane + 32) * w + k], xk, x1);
        x0 = fma(-S.L[lane * w + k], xk, x0);  // lane < 32 <= k
      } else {
        const double xk = __shfl_sync(0xffffffffu, x0, k);
        if (lane < k) x0 = fma(-S.L[lane * w + k], xk, x0);
      }
    }
    if (lane < w) __stcg(x + f + lane, x0);
    if (lane + 32 < w) __stcg(x + f + lane + 32, x1);
  }
}

__global__ void __launch_bounds__(kThreads, 2) k_chol_forward_tasks(CholDev d, CholTasks g,
                                                                     double* __restrict__ y) {
  __shared__ double sL[kCholMaxWidth * kCholMaxWidth], sv[kCholMaxWidth], sdi[kCholMaxWidth],
      sz[kSolveZCap];
  const SolveStage S{sL, sv, sdi, sz};
  task_loop(
      g, d.abort, [&](int4 tk) { return forward_staged_pre(d, tk.y, y, S); },
      [&](int4 tk, const StagedPre& st) {
        if (st.staged)
          forward_staged_run(d, tk.y, y, S, st);
        else
          forward_large(d, tk.y, y, sL, sv);
      });
  wait_prior_grid();
}

__global__ void __launch_bounds__(kThreads, 2) k_chol_backward_tasks(CholDev d, CholTasks g,
                                                                      double* __restrict__ x) {
  // the backward warp tasks may start now: they wait for this kernel's flags
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  __shared__ double sL[kCholMaxWidth * kCholMaxWidth], sv[kCholMaxWidth], sdi[kCholMaxWidth],
      sz[kSolveZCap];
  const SolveStage S{sL, sv, sdi, sz};
  task_loop(
      g, d.abort, [&](int4 tk) { return backward_staged_pre(d, tk.y, x, S); },
      [&](int4 tk, const StagedPre& st) {
        if (st.staged)
          backward_staged_run(d, tk.y, x, S, st);
        else
          backward_large(d, tk.y, x, sL, sv);
      });
}

// Warp tasks: each warp takes the next task of the list, waits (bounded)
// for the tasks it depends on, runs it and sets its flag; the same progress
// argument as task_loop, with warps for blocks.
template <typename Pre, typename Run>
__device__ __forceinline__ void warp_task_loop(const CholTasks& g, int32_t* abort, Pre pre,
                                               Run run) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    int t = 0;
    unsigned long long t0 = 0ull;
    if (lane == 0) {
      t = ld_acquire(abort) ? g.n : atomicAdd(g.next, 1);
      if (g.trace) t0 = gpu_clock_ns();
    }
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= g.n) return;
    const int4 tk = __ldg(g.task + t);
    const auto early = pre(tk);
    bool ok = true;  // the lanes watch the dependencies together
    {
      const int q1 = __ldg(g.dep_ptr + t + 1);
      for (int q = __ldg(g.dep_ptr + t) + lane; q < q1 && ok; q += 32)
        ok = wait_done(g.done + __ldg(g.dep + q), abort);
      if (g.xdep_ptr) {  // tasks of the graph launched before this one
        const int x1 = __ldg(g.xdep_ptr + t + 1);
        for (int q = __ldg(g.xdep_ptr + t) + lane; q < x1 && ok; q += 32)
          ok = wait_done(g.xdone + __ldg(g.xdep + q), abort);
      }
      __syncwarp();  // orders every lane's reads after the lanes' acquires
    }
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) return;
    const unsigned long long t1 = g.trace && lane == 0 ? gpu_clock_ns() : 0ull;
    run(tk, early);
    __syncwarp();  // the lanes' writes before lane 0's release
    if (lane == 0) {
      st_release(g.done + t, 1);
      if (g.trace) {
        long long* r = g.trace + 6 * size_t(t);
        r[0] = tk.x;
        r[1] = tk.y;
        r[2] = (long long)t0;
        r[3] = (long long)t1;
        r[4] = (long long)gpu_clock_ns();
        r[5] = sm_id();
      }
    }
  }
}

// The solves' warp tasks: one small supernode per warp.
template <bool kForward>
__global__ void __launch_bounds__(kThreads) k_chol_solve_warps(CholDev d, CholTasks g,
                                                                double* __restrict__ v) {
  // (forward) the block tasks may start now: they wait for this kernel's flags
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  __shared__ double ws_all[kWarps * (kSmallPanel + kCholWarpRows)];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* ws = ws_all + warp * (kSmallPanel + kCholWarpRows);
  if constexpr (kForward)
    warp_task_loop(
        g, d.abort, [&](int4 tk) { return forward_small_pre(d, tk.y, lane, v, ws); },
        [&](int4, const FwdSmall& st) { forward_small_run(d, st, lane, v, ws); });
  else
    warp_task_loop(
        g, d.abort, [&](int4 tk) { return backward_small_pre(d, tk.y, lane, v, ws); },
        [&](int4, const BwdSmall& st) { backward_small_run(st, lane, v, ws); });
  wait_prior_grid();
}

// The factorization's warp tasks: one warp-small supernode per warp, staged
// in the warp's slice of shared memory (kSmallStage doubles, then its row
// map scratch).
__global__ void __launch_bounds__(kThreads) k_chol_factor_warps(CholDev d, CholTasks g,
                                                                 double tol) {
  // the task kernel after this one may start now: its blocks take SMs as
  // this kernel's blocks leave, and wait for this kernel's flags
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  extern __shared__ double smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* ws = smem + warp * kSmallStage;
  int* wr = reinterpret_cast<int*>(smem + kWarps * kSmallStage) + warp * kCholWarpRows;
  warp_task_loop(g, d.abort, [](int4) { return 0; },
                 [&](int4 tk, int) { factor_staged<32>(d, tk.y, lane, tol, ws, wr); });
}

constexpr size_t kFactorWarpSmem =
    size_t(kWarps) * kSmallStage * sizeof(double) + size_t(kWarps) * kCholWarpRows * sizeof(int);

int grid_for(int64_t n, int threads) {
  return n > 0 ? int(std::min<int64_t>((n + threads - 1) / threads, 4096)) : 0;
}

}  // namespace

cudaError_t launch_gather(double* out, const double* in, const int32_t* idx, int n,
                          cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_gather<<<grid_for(n, kPermThreads), kPermThreads, 0, s>>>(out, in, idx, n);
  return cudaGetLastError();
}

cudaError_t launch_scatter(double* out, const double* in, const int32_t* idx, int n,
                           cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_scatter<<<grid_for(n, kPermThreads), kPermThreads, 0, s>>>(out, in, idx, n);
  return cudaGetLastError();
}

cudaError_t launch_chol_assemble(double* Lx, const int64_t* amap, const double* kvals,
                                 int64_t nnz, cudaStream_t s) {
  if (nnz <= 0) return cudaSuccess;
  k_chol_assemble<<<grid_for(nnz, kPermThreads), kPermThreads, 0, s>>>(Lx, amap, kvals, nnz);
  return cudaGetLastError();
}

size_t chol_bottom_smem_bytes(int stage) {
  return size_t(kBotMap + stage) * kBotThreads * sizeof(double);
}

cudaError_t launch_chol_bottom(const CholDev& d, const int32_t* list, int count, int stage,
                               double tol, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_chol_bottom<<<(count + kBotThreads - 1) / kBotThreads, kBotThreads,
                  chol_bottom_smem_bytes(stage), s>>>(d, list, count, tol);
  return cudaGetLastError();
}

cudaError_t launch_chol_bottom_fwd(const CholDev& d, const int32_t* list, int count, double* y,
                                   cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_chol_bottom_fwd<<<(count + kThreads - 1) / kThreads, kThreads, 0, s>>>(d, list, count, y);
  return cudaGetLastError();
}

cudaError_t launch_chol_bottom_bwd(const CholDev& d, const int32_t* list, int count, double* x,
                                   cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_chol_bottom_bwd<<<(count + kThreads - 1) / kThreads, kThreads, 0, s>>>(d, list, count, x);
  return cudaGetLastError();
}

size_t chol_task_smem_bytes() {
  return size_t(kStageDoubles) * sizeof(double) + size_t(kRelInts) * sizeof(int);
}

cudaError_t chol_task_setup(int* blocks_per_sm, int* warp_blocks_per_sm) {
  const size_t bytes = chol_task_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_chol_factor_tasks,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
  int per_sm = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chol_factor_tasks, kThreads, bytes);
  if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_chol_bottom, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(chol_bottom_smem_bytes(kCholBottomStage)));
  if (e == cudaSuccess) *blocks_per_sm = std::min(per_sm, 2);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_chol_factor_warps, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(kFactorWarpSmem));
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chol_factor_warps, kThreads,
                                                      kFactorWarpSmem);
  if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
  if (e == cudaSuccess) *warp_blocks_per_sm = per_sm;
  return e;
}

cudaError_t launch_chol_factor_warps(const CholDev& d, const CholTasks& t, double tol, int blocks,
                                     cudaStream_t s) {
  if (t.n <= 0) return cudaSuccess;
  const int grid = std::min(blocks, (t.n + kWarps - 1) / kWarps);
  k_chol_factor_warps<<<grid, kThreads, kFactorWarpSmem, s>>>(d, t, tol);
  return cudaGetLastError();
}

cudaError_t launch_chol_factor_tasks(const CholDev& d, const CholTasks& t, double tol, int blocks,
                                     bool early, cudaStream_t s) {
  if (t.n <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(std::min(blocks, t.n)));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = chol_task_smem_bytes();
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = early ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k_chol_factor_tasks, d, t, tol);
}

// Launches kern with programmatic dependent launch when `early`: it may start
// once every block of the kernel before it has started (each triggers at its
// first instruction), and it waits for that kernel's tasks through flags.
template <typename Kern, typename... Args>
cudaError_t launch_early(Kern kern, int grid, bool early, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = early ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

cudaError_t launch_chol_forward_tasks(const CholDev& d, const CholTasks& t, double* y, int blocks,
                                      bool early, cudaStream_t s) {
  if (t.n <= 0) return cudaSuccess;
  return launch_early(k_chol_forward_tasks, std::min(blocks, t.n), early, s, d, t, y);
}

cudaError_t launch_chol_backward_tasks(const CholDev& d, const CholTasks& t, double* x, int blocks,
                                       cudaStream_t s) {
  if (t.n <= 0) return cudaSuccess;
  k_chol_backward_tasks<<<std::min(blocks, t.n), kThreads, 0, s>>>(d, t, x);
  return cudaGetLastError();
}

cudaError_t launch_chol_solve_warps(const CholDev& d, const CholTasks& t, double* v, bool forward,
                                    int blocks, bool early, cudaStream_t s) {
  if (t.n <= 0) return cudaSuccess;
  const int grid = std::min(blocks, (t.n + kWarps - 1) / kWarps);
  if (forward) return launch_early(k_chol_solve_warps<true>, grid, early, s, d, t, v);
  return launch_early(k_chol_solve_warps<false>, grid, early, s, d, t, v);
}

}  // namespace acopf
