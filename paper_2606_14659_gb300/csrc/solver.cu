// solver.cu — Fiedler solvers of librsb, batched over all units of a level.
//
// Lanczos with restarts (paper §6), the Lanczos vectors kept orthonormal by
// classical Gram-Schmidt with a second pass (CGS2).  FP64 steps:
//   A: w = L q_j, fused with the first Gram-Schmidt pass's dot products
//      against [1/sqrt(n), deflation vectors, q_0..q_j],
//   B: w -= basis * c1, fused with the second pass's dot products,
//   C: w -= basis * c2, fused with ||w||^2 -> beta_{j+1};
// q_{j+1} = w / beta_{j+1} is materialised by the next step's A, which gathers
// the unnormalised w and scales.  FP32 steps (bandwidth-bound) delay the
// second pass by one step, two passes over the basis instead of three:
//   D1: z = L v_j (v_j = w_j / nu_j, projected once),
//   D2: a = B^T v_j, g = B^T z, v.v, v.z in one pass -> q_j = (v_j - B a) / rho
//       and column j of S,
//   D3: q_j and w_{j+1} = (z - B g - (q_j.z) q_j) / rho in one pass, nu_{j+1}.
// After the cycle: the Ritz pairs of the
// projected matrix S = Q^T L Q (parallel cyclic Jacobi, one CTA per unit), the
// Ritz vector y = Q t, the true residual ||L y - theta y||, and a thick restart
// from the kept Ritz vectors and the last residual direction (an explicit
// restart from y, projected against the fixed basis, when a cycle ended on an
// invariant subspace).  Launch modes: one kernel per step phase (optionally
// replayed as a CUDA graph per cycle), one cooperative kernel per cycle (CGS2
// in both precisions), or one cooperative kernel per solve with the basis
// resident in shared memory (the steps of the per-phase kernels, bit for bit).
//
// Inverse iteration (paper §7, Algorithm 2): the right-hand side b is the
// projected, normalised previous iterate; L x = b is solved by CG from x0 = 0
// with r projected against the fixed basis every step; the Rayleigh quotient
// and residual of x decide the stop (also when CG returned after a single
// iteration, §7).
//
// Precision: V = double (plain FP64) or V = float (vectors, SpMV and updates
// in FP32; per-thread Kahan sums in FP32; CTA and cross-CTA sums, the
// Gram-Schmidt coefficients, T, and the CG alpha/beta recurrences in FP64).
#include <chrono>
#include <algorithm>
#include <cfloat>

#include "rsb_internal.cuh"

int g_rsb_poison_barrier = 0;  // test hook, see rsb_test_poison_barrier

template <typename V>
struct LzArgs {
  const int64_t* slice_ptr;
  const uint32_t* ent;
  const int64_t* gid;
  const Tile* tiles;
  Unit* units;
  const uint64_t* ckey;
  V* Q;
  long long N;
  V* W0;
  V* W1;
  V* Y;
  V* X;
  V* R;
  V* P;
  V* AP;
  const double* D0;
  const double* D1;
  double* partials;
  long long stride;
  int* n_active;
  long long* stat_cycles;
  unsigned long long* pb_a;  // profiling byte counters (nullptr when off)
  unsigned long long* pb_a2;
  unsigned long long* pb_b;
  unsigned long long* pb_c;
  unsigned long long* pb_cg;
  double* S;                 // per unit: projected matrix S (M x M) then Ritz vectors Y
  int* jmin;                 // smallest first step of the next cycle over the units
};

// CTA-level add of per-thread byte counts to a profiling counter.
__device__ __forceinline__ void prof_add(unsigned long long* pb, unsigned long long b) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(pb, b);
}

__device__ __forceinline__ int row_width(const int64_t* __restrict__ slice_ptr, int r) {
  return (int)((slice_ptr[(r >> 5) + 1] - slice_ptr[r >> 5]) >> 5);
}

template <typename V, bool CO = false>
__device__ __forceinline__ V spmv_row(const int64_t* __restrict__ slice_ptr,
                                      const uint32_t* __restrict__ ent, const V* x, int r, V xr) {
  const int64_t base = slice_ptr[r >> 5];
  const int width = (int)((slice_ptr[(r >> 5) + 1] - base) >> 5);
  const uint32_t* e = ent + base + (r & 31);
  V acc = V(0);
  uint32_t dsum = 0;
#pragma unroll 4
  for (int k = 0; k < width; ++k) {
    const uint32_t p = __ldg(e + 32 * k);
    if constexpr (sizeof(V) == 8) {  // FP64: d_r x_r - sum w x_c, as spmv_row_ro
      acc = fma(weight_f64(ent_w(p)), ldc<CO>(x + ent_col(p)), acc);
      dsum += ent_w(p);
    } else {
      acc += V(ent_w(p)) * (xr - ldc<CO>(x + ent_col(p)));
    }
  }
  if constexpr (sizeof(V) == 8) return fma((double)dsum, xr, -acc);
  return acc;
}

// ----------------------------------------------------------------------------
// Gram-Schmidt building blocks.  The basis is [u0, D_0.., q_0..q_j] with
// u0 = 1/sqrt(n) on unit rows (its dot is taken as a plain sum and scaled by
// 1/sqrt(n) afterwards).  A CTA handles its tile in sub-chunks of up to
// RSB_BLOCK * RSB_SUBR rows: phase 1 computes the chunk's w (one row per
// thread and RSB_SUBR rows per thread, coefficient-outer so that every
// thread has RSB_SUBR independent loads in flight), stores it in shared
// memory; phase 2 takes the dot products warp-per-coefficient with unrolled
// coalesced loads.
// ----------------------------------------------------------------------------
#define MAXCW ((RSB_MAXC + RSB_WARPS - 1) / RSB_WARPS)
#define SUBROWS (RSB_BLOCK * RSB_SUBR)

// Warp-per-coefficient dots of basis coefficients [c0, c0 + nc) with the chunk:
// warp w owns coefficients w, w + 8, ...; each lane walks rows in groups of 4
// and issues the loads of all of its warp's coefficients for the group before
// accumulating, so up to 4 * MAXCW loads are in flight per lane.
template <typename V>
__device__ __forceinline__ void tile_dots(const LzArgs<V>& a, int nd, int c0, int nc, int base,
                                          int end, const V* ws, Acc<V> (&acc)[MAXCW]) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const V* qp[MAXCW];
  const double* dp[MAXCW];
  int kind[MAXCW];  // -1 none, 0 ones (u0), 1 FP64 deflation vector, 2 basis vector
#pragma unroll
  for (int i = 0; i < MAXCW; ++i) {
    const int c = w + RSB_WARPS * i;
    const int cc = c0 + c;
    qp[i] = nullptr;
    dp[i] = nullptr;
    if (c >= nc) kind[i] = -1;
    else if (cc == 0) kind[i] = 0;
    else if (cc <= nd) {
      kind[i] = 1;
      dp[i] = cc == 1 ? a.D0 : a.D1;
    } else {
      kind[i] = 2;
      qp[i] = a.Q + (long long)(cc - 1 - nd) * a.N;
    }
  }
  if (kind[0] < 0) return;
  for (int row = base + lane; row < end; row += 128) {
    V wv[4];
    bool ok[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      ok[q] = row + 32 * q < end;
      wv[q] = ok[q] ? ws[row + 32 * q - base] : V(0);
    }
    V b[MAXCW][4];
#pragma unroll
    for (int i = 0; i < MAXCW; ++i)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = row + 32 * q;
        b[i][q] = V(0);
        if (ok[q]) {
          if (kind[i] == 2) b[i][q] = qp[i][r];
          else if (kind[i] == 1) b[i][q] = V(dp[i][r]);
          else if (kind[i] == 0) b[i][q] = V(1);
        }
      }
#pragma unroll
    for (int i = 0; i < MAXCW; ++i)
      if (kind[i] >= 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (ok[q]) acc[i].add(b[i][q] * wv[q]);
      }
  }
}

template <typename V>
__device__ __forceinline__ void store_dots(const LzArgs<V>& a, int nc, Acc<V> (&acc)[MAXCW],
                                           int tix) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < MAXCW; ++i) {
    const int c = w + RSB_WARPS * i;
    if (c < nc) {
      const double s = warp_total(acc[i]);
      if (lane == 0) a.partials[(long long)c * a.stride + tix] = s;
    }
  }
}

// w[rr] -= sum_c cv[c] basis_c for the RSB_SUBR rows of this thread
// (rows base + rr*RSB_BLOCK + tid), coefficient-outer; cv holds the
// coefficients already in the vector type (stage_coef).
template <typename V, bool CO>
__device__ __forceinline__ void gs_update_rows(const LzArgs<V>& a, const Unit& u, const V* cv,
                                               int nd, int nq, int base, int end,
                                               V (&w)[RSB_SUBR]) {
  const V c0 = cv[0];
#pragma unroll
  for (int rr = 0; rr < RSB_SUBR; ++rr) {
    const int r = base + rr * RSB_BLOCK + threadIdx.x;
    if (r < end && unit_has(u, a.ckey, r)) w[rr] -= c0;
  }
  for (int l = 0; l < nd; ++l) {
    const double* d = l == 0 ? a.D0 : a.D1;
    const V cl = cv[1 + l];
#pragma unroll
    for (int rr = 0; rr < RSB_SUBR; ++rr) {
      const int r = base + rr * RSB_BLOCK + threadIdx.x;
      if (r < end) w[rr] -= cl * V(d[r]);
    }
  }
  const V* cq = cv + 1 + nd;
  bool ok[RSB_SUBR];
#pragma unroll
  for (int rr = 0; rr < RSB_SUBR; ++rr) ok[rr] = base + rr * RSB_BLOCK + (int)threadIdx.x < end;
  int k = 0;
  for (; k + 4 <= nq; k += 4) {  // four basis vectors per round: 4 * RSB_SUBR loads in flight
    V qv[4][RSB_SUBR];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const V* q = a.Q + (long long)(k + i) * a.N + base + threadIdx.x;
#pragma unroll
      for (int rr = 0; rr < RSB_SUBR; ++rr) qv[i][rr] = ok[rr] ? q[rr * RSB_BLOCK] : V(0);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const V ck = cq[k + i];
#pragma unroll
      for (int rr = 0; rr < RSB_SUBR; ++rr) w[rr] -= ck * qv[i][rr];
    }
  }
  for (; k < nq; ++k) {
    const V ck = cq[k];
    const V* q = a.Q + (long long)k * a.N + base + threadIdx.x;
#pragma unroll
    for (int rr = 0; rr < RSB_SUBR; ++rr)
      if (ok[rr]) w[rr] -= ck * q[rr * RSB_BLOCK];
  }
}

// ----------------------------------------------------------------------------
// Lanczos step (thick-restarted, full re-orthogonalisation): per-tile bodies
// (CO = running inside the persistent cycle kernel, where data written by
// other CTAs earlier in the launch is read through L2) and the stand-alone
// kernels that wrap them.
//   A(j): q_j = src / beta (src is the unnormalised new vector), w = L q_j,
//         first Gram-Schmidt pass coefficients c1 = [1, D, q_0..q_j]^T w;
//   B(j): w -= basis c1, second-pass coefficients c2; column j of the
//         projected matrix S = Q^T L Q is c1 + c2 on q_0..q_j;
//   C(j): w -= basis c2, beta_{j+1} = ||w|| (w stays unnormalised for A(j+1)).
// ----------------------------------------------------------------------------
__device__ __forceinline__ double* unit_S(double* S, int ui) { return S + (long long)ui * RSB_SSTRIDE; }

template <typename V, bool CO>
__device__ __forceinline__ void lz_a_t(const LzArgs<V>& a, int j, int tix, V* ws, double* out) {
  const Tile t = a.tiles[tix];
  Unit& u = a.units[t.unit];
  if (ldc<CO>(&u.status) != U_ACTIVE || j >= ldc<CO>(&u.msteps) || j < ldc<CO>(&u.j0)) return;
  const V* src = (j & 1) ? a.W1 : a.W0;
  V* dst = (j & 1) ? a.W0 : a.W1;
  V* qj = a.Q + (long long)j * a.N;
  // 1 / beta once per CTA (an FP64 division per thread costs the SM's FP64 pipe)
  if (threadIdx.x == 0)
    out[0] = 1.0 / (j == ldc<CO>(&u.j0) ? ldc<CO>(&u.beta0) : ldc<CO>(&u.beta[j]));
  __syncthreads();
  const V s = V(out[0]);
  const int nd = u.nd;
  const int nc = 2 + nd + j;
  Acc<V> acc[MAXCW];
  unsigned long long pbytes = 0;
  for (int base = t.row0; base < t.row1; base += SUBROWS) {
    const int end = min(t.row1, base + SUBROWS);
#pragma unroll 2
    for (int rr = 0; rr < RSB_SUBR; ++rr) {
      const int r = base + rr * RSB_BLOCK + threadIdx.x;
      V w = V(0);
      if (r < end) {
        const V xr = src[r];
        w = s * spmv_row<V, CO>(a.slice_ptr, a.ent, src, r, xr);
        qj[r] = s * xr;
        dst[r] = w;
        if (a.pb_a)
          pbytes += 4ull * row_width(a.slice_ptr, r) +
                    sizeof(V) * (unsigned long long)(4 + j) + 8ull * nd;
      }
      ws[rr * RSB_BLOCK + threadIdx.x] = w;
    }
    __syncthreads();
    tile_dots<V>(a, nd, 0, nc, base, end, ws, acc);
    __syncthreads();
  }
  store_dots<V>(a, nc, acc, tix);
  if (a.pb_a) prof_add(a.pb_a, pbytes);
  if (last_cta(&u.cnt, u.ntile)) {
    final_reduce(a.partials, a.stride, u.tile0, u.ntile, nc, out);
    if (threadIdx.x == 0) {
      u.c1[0] = out[0] * u.isn;
      for (int c = 1; c < nc; ++c) u.c1[c] = out[c];
    }
  }
}

template <typename V, bool CO>
__device__ __forceinline__ void lz_b_t(const LzArgs<V>& a, int j, int tix, V* ws, V* cv,
                                       double* out) {
  const Tile t = a.tiles[tix];
  Unit& u = a.units[t.unit];
  if (ldc<CO>(&u.status) != U_ACTIVE || j >= ldc<CO>(&u.msteps) || j < ldc<CO>(&u.j0)) return;
  V* w_ = (j & 1) ? a.W0 : a.W1;
  const int nd = u.nd;
  const int nc = 2 + nd + j;
  stage_coef<V, CO>(u.c1, nc, u.isn, cv);
  Acc<V> acc[MAXCW];
  unsigned long long pbytes = 0;
  for (int base = t.row0; base < t.row1; base += SUBROWS) {
    const int end = min(t.row1, base + SUBROWS);
    V w[RSB_SUBR];
#pragma unroll
    for (int rr = 0; rr < RSB_SUBR; ++rr) {
      const int r = base + rr * RSB_BLOCK + threadIdx.x;
      w[rr] = r < end ? w_[r] : V(0);
    }
    gs_update_rows<V, CO>(a, u, cv, nd, j + 1, base, end, w);
#pragma unroll
    for (int rr = 0; rr < RSB_SUBR; ++rr) {
      const int r = base + rr * RSB_BLOCK + threadIdx.x;
      if (r < end) {
        w_[r] = w[rr];
        if (a.pb_b) pbytes += sizeof(V) * (unsigned long long)(3 + j) + 8ull * nd;
      }
      ws[rr * RSB_BLOCK + threadIdx.x] = r < end ? w[rr] : V(0);
    }
    __syncthreads();
    tile_dots<V>(a, nd, 0, nc, base, end, ws, acc);
    __syncthreads();
  }
  store_dots<V>(a, nc, acc, tix);
  if (a.pb_b) prof_add(a.pb_b, pbytes);
  if (last_cta(&u.cnt, u.ntile)) {
    final_reduce(a.partials, a.stride, u.tile0, u.ntile, nc, out);
    if (threadIdx.x == 0) {
      u.c2[0] = out[0] * u.isn;
      for (int c = 1; c < nc; ++c) u.c2[c] = out[c];
    }
    __syncthreads();
    double* Sm = unit_S(a.S, t.unit);
    for (int k = threadIdx.x; k <= j; k += RSB_BLOCK) {
      const double v = ldc<CO>(&u.c1[1 + nd + k]) + out[1 + nd + k];
      Sm[k * RSB_MAXM + j] = v;
      Sm[j * RSB_MAXM + k] = v;
    }
  }
}

template <typename V, bool CO>
__device__ __forceinline__ void lz_c_t(const LzArgs<V>& a, int j, double breakdown, int tix,
                                       V* cv, double* sm, double* out) {
  const Tile t = a.tiles[tix];
  Unit& u = a.units[t.unit];
  if (ldc<CO>(&u.status) != U_ACTIVE || j >= ldc<CO>(&u.msteps) || j < ldc<CO>(&u.j0)) return;
  V* w_ = (j & 1) ? a.W0 : a.W1;
  const int nd = u.nd;
  stage_coef<V, CO>(u.c2, 2 + nd + j, u.isn, cv);
  Acc<V> acc;
  unsigned long long pbytes = 0;
  for (int base = t.row0; base < t.row1; base += SUBROWS) {
    const int end = min(t.row1, base + SUBROWS);
    V w[RSB_SUBR];
#pragma unroll
    for (int rr = 0; rr < RSB_SUBR; ++rr) {
      const int r = base + rr * RSB_BLOCK + threadIdx.x;
      w[rr] = r < end ? w_[r] : V(0);
    }
    gs_update_rows<V, CO>(a, u, cv, nd, j + 1, base, end, w);
#pragma unroll
    for (int rr = 0; rr < RSB_SUBR; ++rr) {
      const int r = base + rr * RSB_BLOCK + threadIdx.x;
      if (r < end) {
        w_[r] = w[rr];
        acc.add(w[rr] * w[rr]);
        if (a.pb_c) pbytes += sizeof(V) * (unsigned long long)(3 + j) + 8ull * nd;
      }
    }
  }
  if (a.pb_c) prof_add(a.pb_c, pbytes);
  const double sum = block_total(acc, sm);
  if (threadIdx.x == 0) a.partials[tix] = sum;
  if (last_cta(&u.cnt, u.ntile)) {
    final_reduce(a.partials, a.stride, u.tile0, u.ntile, 1, out);
    if (threadIdx.x == 0) {
      const double b = sqrt(out[0]);
      u.beta[j + 1] = b;
      if (b <= breakdown * u.dmax) {  // invariant subspace: the cycle ends here
        u.msteps = j + 1;
        u.broke = 1;
      }
    }
  }
}

template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK, sizeof(V) == 4 ? 3 : 2) k_lz_a(LzArgs<V> a, int j) {
  __shared__ V ws[SUBROWS];
  __shared__ double out[RSB_MAXC];
  lz_a_t<V, false>(a, j, blockIdx.x, ws, out);
}

template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK, sizeof(V) == 4 ? 3 : 2) k_lz_b(LzArgs<V> a, int j) {
  __shared__ V ws[SUBROWS];
  __shared__ V cv[RSB_MAXC];
  __shared__ double out[RSB_MAXC];
  lz_b_t<V, false>(a, j, blockIdx.x, ws, cv, out);
}

template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_lz_c(LzArgs<V> a, int j, double breakdown) {
  __shared__ double sm[RSB_WARPS];
  __shared__ V cv[RSB_MAXC];
  __shared__ double out[1];
  lz_c_t<V, false>(a, j, breakdown, blockIdx.x, cv, sm, out);
}

// ----------------------------------------------------------------------------
// Bulk-copy staging (launch modes 0 and 1, FP32 step D2).  The tile is walked
// in chunks of ST_CH rows; for every chunk one thread issues 1-D bulk copies
// (cp.async.bulk, completion counted in bytes on an mbarrier) of the chunk's
// rows of the basis (and of the step's work vectors) into shared memory, one
// chunk ahead of the one being computed.  Waits on the mbarrier are bounded
// (2 s of the global timer): on timeout the CTA sets the grid error word, waits
// (bounded) for its own copies still in flight and returns.
// ----------------------------------------------------------------------------
// The staged kernels walk a tile in chunks of ST_CH rows through ST_NB
// buffers: while a chunk is being computed, the next ST_NB - 1 chunks are in
// flight.  Thread 0 issues the copies of a chunk, one per basis vector.
// (Measured slower on GB300: four buffers of 128 rows for the same shared
// memory, twice the copies for the same bytes; the copies issued by the 32
// lanes of a warp together; and an L2 bulk prefetch of the chunks two ahead of
// the copies.)
#define ST_CH 256
#define ST_NB 2

template <typename V>
struct BulkRows {
  static constexpr int AL = 16 / sizeof(V);        // rows per 16 bytes
  static constexpr int CRB = ST_CH + AL;           // staged rows per vector and buffer
};

template <typename V>
constexpr size_t staged_smem(int nq) {
  return ST_NB * (size_t)nq * BulkRows<V>::CRB * sizeof(V);
}

// Wait for chunk ci (buffer ci % ST_NB); false (uniform) when the copies did
// not complete in time, after flagging the grid error word and draining this
// CTA's copies still in flight (chunks ci .. ci + ST_NB - 1).
__device__ __forceinline__ bool staged_wait(uint64_t* bar, int ci, int nchunk, GridBar* gb) {
  const bool ok = mbar_wait_bounded(&bar[ci % ST_NB], (ci / ST_NB) & 1, 2000000000ull);
  if (!__syncthreads_or(!ok)) return true;
  if (threadIdx.x == 0) {
    atomicMax(&gb->err, 1);
    bool drained = true;
    for (int c = ci; c < min(nchunk, ci + ST_NB); ++c)
      drained = mbar_wait_bounded(&bar[c % ST_NB], (c / ST_NB) & 1, 1000000000ull) && drained;
    if (!drained) atomicMax(&gb->err, 2);
  }
  __syncthreads();
  return false;
}

// Thread 0: rows [c0, c1) of q_0..q_{nq-1} (rounded out to 16 bytes) into
// buffer b of Qb ([ST_NB][slots][CRB]), completing on bar[b].
// (extra and extra2, when given, are N-vectors staged after q_{nq-1}; slots =
// nq plus the extras given)
template <typename V>
__device__ __forceinline__ void bulk_issue_chunk(const LzArgs<V>& a, V* Qb, uint64_t* bar, int nq,
                                                 int b, int c0, int c1,
                                                 const V* extra = nullptr,
                                                 const V* extra2 = nullptr) {
  constexpr int AL = BulkRows<V>::AL, CRB = BulkRows<V>::CRB;
  const int slots = nq + (extra ? 1 : 0) + (extra2 ? 1 : 0);
  const int a0 = c0 & ~(AL - 1);
  const int len = (c1 - a0 + AL - 1) / AL * AL;
  const unsigned bytes = (unsigned)(len * sizeof(V));
  V* dst = Qb + (size_t)b * slots * CRB;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_expect_tx(&bar[b], bytes * (unsigned)slots);
  for (int k = 0; k < nq; ++k)
    bulk_g2s(dst + (size_t)k * CRB, a.Q + (long long)k * a.N + a0, bytes, &bar[b]);
  int k = nq;
  if (extra) bulk_g2s(dst + (size_t)(k++) * CRB, extra + a0, bytes, &bar[b]);
  if (extra2) bulk_g2s(dst + (size_t)k * CRB, extra2 + a0, bytes, &bar[b]);
}

// Thread 0 of a staged kernel: the copies of chunk c into its buffer.
template <typename V>
__device__ __forceinline__ void stage_chunk(const LzArgs<V>& a, V* Qb, uint64_t* bar, int nq,
                                            const Tile& t, int c, const V* extra = nullptr,
                                            const V* extra2 = nullptr) {
  const int n0 = t.row0 + c * ST_CH;
  bulk_issue_chunk(a, Qb, bar, nq, c % ST_NB, n0, min(t.row1, n0 + ST_CH), extra, extra2);
}

// Step D1 of the FP32 streaming path: z = L (src / nu_j) into the work vector
// AP (src stays as it is: D2 and D3 read it).  A CTA takes A1_RPT * RSB_BLOCK consecutive rows of a tile (CTA b: tile
// b / nsub, part b % nsub of it), A1_RPT rows per thread.
#ifndef A1_RPT
#define A1_RPT 4
#endif
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_lz_a1(LzArgs<V> a, int j, int nsub) {
  __shared__ double scale;
  const int tix = (int)(blockIdx.x / (unsigned)nsub);
  const Tile t = a.tiles[tix];
  const long long p0 = (long long)t.row0 +
                       (long long)(blockIdx.x - (unsigned)tix * nsub) * (A1_RPT * RSB_BLOCK);
  if (p0 >= t.row1) return;
  const int p1 = (int)min((long long)t.row1, p0 + A1_RPT * RSB_BLOCK);
  const Unit& u = a.units[t.unit];
  if (u.status != U_ACTIVE || j >= u.msteps || j < u.j0) return;
  if (threadIdx.x == 0) scale = 1.0 / (j == u.j0 ? u.beta0 : u.beta[j]);
  __syncthreads();
  const V s = V(scale);
  const V* src = (j & 1) ? a.W1 : a.W0;
  V* z = a.AP;
  unsigned long long pbytes = 0;
#pragma unroll 4
  for (int r = (int)p0 + threadIdx.x; r < p1; r += RSB_BLOCK) {
    const V xr = src[r];
    z[r] = s * spmv_row_ro<V>(a.slice_ptr, a.ent, src, r, xr);
    if (a.pb_a) pbytes += 4ull * row_width(a.slice_ptr, r) + 2ull * sizeof(V);
  }
  if (a.pb_a) prof_add(a.pb_a, pbytes);
}

// Closing arithmetic of step D2 for one unit (every thread of the CTA takes
// part), from the reduced totals av = [a_b (b < nb), v.v] and gz = [g_b
// (b < nb), v.z] of src, scaled here in place to v = src / nu (inu = 1 / nu)
// and u0 = 1/sqrt(n) on its entry; sc[0..2] = rho, q_j.z, alpha and
// sk[0..j) = S_kj come back in shared memory.  S is read for columns < j;
// column and row j are written when write_s.  The streaming kernel and the
// resident kernel both call this, so both modes produce the same numbers.
template <bool CO>
__device__ void d2_finish(double* av, double* gz, int nb, int nd, int j, double inu, double isn,
                          double* Sm, bool write_s, double* sc, double* sk) {
  if (threadIdx.x == 0) {
    for (int b = 0; b < nb; ++b) av[b] *= inu;
    av[nb] *= inu * inu;
    gz[nb] *= inu;
    av[0] *= isn;
    gz[0] *= isn;
    double aa = 0.0, ag = 0.0;
    for (int b = 0; b < nb; ++b) {
      aa += av[b] * av[b];
      ag += av[b] * gz[b];
    }
    const double rho2 = av[nb] - aa;
    // v has unit norm and |a| is at rounding level after its first pass; a
    // non-positive rho^2 means v lies in span(B) to working precision
    const double rho = rho2 > 0.0 ? sqrt(rho2) : 1e-300;
    sc[0] = rho;
    sc[1] = (gz[nb] - ag) / rho;  // q_j.z
  }
  __syncthreads();
  const double rho = sc[0];
  const double* aq = av + 1 + nd;  // a on q_0..q_{j-1}
  for (int k = threadIdx.x; k < j; k += RSB_BLOCK) {
    double sa_k = 0.0;
    for (int i = 0; i < j; ++i) sa_k += ldc<CO>(Sm + k * RSB_MAXM + i) * aq[i];
    sk[k] = (gz[1 + nd + k] - sa_k) / rho;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sig = 0.0;
    for (int k = 0; k < j; ++k) sig += sk[k] * aq[k];
    sc[2] = (sc[1] - sig) / rho;
    if (write_s) Sm[j * RSB_MAXM + j] = sc[2];
  }
  if (write_s)
    for (int k = threadIdx.x; k < j; k += RSB_BLOCK) {
      Sm[k * RSB_MAXM + j] = sk[k];
      Sm[j * RSB_MAXM + k] = sk[k];
    }
  __syncthreads();
}

// ----------------------------------------------------------------------------
// Step D2 of the FP32 streaming path (second Gram-Schmidt pass delayed by one
// step, DCGS2: Swirydowicz, Langou, Ananthan, Yang and Thomas, "Low
// synchronization Gram-Schmidt and GMRES algorithms", 2020).  v = src / nu_j
// has been projected once against B = [u0, D, q_0..q_{j-1}]; z = L v (D1).
// One staged pass over q_0..q_{j-1}, src and z takes a = B^T v, g = B^T z,
// v.v and v.z; the unit's last CTA then forms
//   rho = sqrt(v.v - a.a)                  q_j = (v - B a) / rho
//   L q_j = (z - L B a) / rho, where L B a lies in span(B, q_j) up to
//   rounding (L u0 = 0; D holds eigenvector approximations; L q_i for i < j
//   is in span(q_0..q_j) by the Lanczos relation), so that
//   S_kj = q_k.L q_j = (g_k - sum_i S_ki a_i) / rho           (k < j)
//   S_jj = (q_j.z - sum_k S_kj a_k) / rho, q_j.z = (v.z - a.g) / rho,
// and the coefficients of D3.  Partials: [a_b (b < nb), v.v] then
// [g_b (b < nb), v.z], nb = 1 + nd + j.
// ----------------------------------------------------------------------------
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK, 4) k_lz_d2(LzArgs<V> a, int j, GridBar* gb) {
  extern __shared__ __align__(128) unsigned char d2_sh[];
  constexpr int AL = BulkRows<V>::AL, CRB = BulkRows<V>::CRB;
  __shared__ __align__(8) uint64_t bar[ST_NB];
  __shared__ double out[2 * RSB_MAXC + 2];
  const Tile t = a.tiles[blockIdx.x];
  Unit& u = a.units[t.unit];
  if (u.status != U_ACTIVE || j >= u.msteps || j < u.j0) return;
  V* Qb = reinterpret_cast<V*>(d2_sh);  // [ST_NB][j + 2][CRB]: q_0..q_{j-1}, src, z
  const int nd = u.nd;
  const int nb = 1 + nd + j;  // columns of B
  const int nc = nb + 1;      // plus v itself (v.v, v.z)
  const int nq = j;
  const int slots = nq + 2;
  const V* src = (j & 1) ? a.W1 : a.W0;
  const int nchunk = (t.row1 - t.row0 + ST_CH - 1) / ST_CH;
  if (threadIdx.x == 0) {
    for (int b = 0; b < ST_NB; ++b) mbar_init(&bar[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int c = 0; c < min(nchunk, ST_NB - 1); ++c)
      bulk_issue_chunk(a, Qb, bar, nq, c, t.row0 + c * ST_CH,
                       min(t.row1, t.row0 + (c + 1) * ST_CH), src, (const V*)a.AP);
  Acc<V> av[MAXCW], az[MAXCW];
  unsigned long long pbytes = 0;
  for (int ci = 0; ci < nchunk; ++ci) {
    if (threadIdx.x == 0 && ci + ST_NB - 1 < nchunk)
      stage_chunk(a, Qb, bar, nq, t, ci + ST_NB - 1, src, (const V*)a.AP);
    if (!staged_wait(bar, ci, nchunk, gb)) return;
    const int c0 = t.row0 + ci * ST_CH;
    const int c1 = min(t.row1, c0 + ST_CH);
    const V* Qc = Qb + (size_t)(ci % ST_NB) * slots * CRB + (c0 - (c0 & ~(AL - 1)));
    const V* vs = Qc + (size_t)nq * CRB;
    const V* zs = vs + CRB;
    const int nr = c1 - c0;
    if (a.pb_a2 && (int)threadIdx.x < nr)
      pbytes += sizeof(V) * (unsigned long long)(2 + j) + 8ull * nd;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < MAXCW; ++i) {
      const int c = w + RSB_WARPS * i;
      if (c < nc) {
        if (c == 0) {
          for (int rl = lane; rl < nr; rl += 32) {
            av[i].add(vs[rl]);
            az[i].add(zs[rl]);
          }
        } else if (c <= nd) {
          const double* d = c == 1 ? a.D0 : a.D1;
          for (int rl = lane; rl < nr; rl += 32) {
            const V dv = V(d[c0 + rl]);
            av[i].add(dv * vs[rl]);
            az[i].add(dv * zs[rl]);
          }
        } else {
          const V* q = c < nb ? Qc + (size_t)(c - 1 - nd) * CRB : vs;
          for (int rl = lane; rl < nr; rl += 32) {
            const V qv = q[rl];
            av[i].add(qv * vs[rl]);
            az[i].add(qv * zs[rl]);
          }
        }
      }
    }
    __syncthreads();
  }
  store_dots<V>(a, nc, av, blockIdx.x);
  {
    LzArgs<V> a2 = a;
    a2.partials = a.partials + (long long)nc * a.stride;
    store_dots<V>(a2, nc, az, blockIdx.x);
  }
  if (a.pb_a2) prof_add(a.pb_a2, pbytes);
  if (last_cta(&u.cnt, u.ntile)) {
    final_reduce(a.partials, a.stride, u.tile0, u.ntile, nc, out);
    final_reduce(a.partials + (long long)nc * a.stride, a.stride, u.tile0, u.ntile, nc, out + nc);
    const double inu = 1.0 / (j == u.j0 ? u.beta0 : u.beta[j]);
    __shared__ double sc[3], sk[RSB_MAXM];
    d2_finish<false>(out, out + nc, nb, nd, j, inu, u.isn, unit_S(a.S, t.unit), true, sc, sk);
    const double rho = sc[0];
    if (threadIdx.x == 0) {
      u.alpha[j] = sc[2];
      // D3: q_j = src / (nu rho) - sum_b (a_b / rho) b,
      //     w = z / rho - sum_b (g_b / rho) b - (q_j.z / rho) q_j
      u.dz_src = inu / rho;
      u.dz_z = 1.0 / rho;
      u.dz_qz = sc[1] / rho;
    }
    for (int b = threadIdx.x; b < nb; b += RSB_BLOCK) {
      u.c2[b] = out[b] / rho;
      u.c1[b] = out[nc + b] / rho;
    }
  }
}

// Step D3 of the FP32 streaming path: per row, q_j = src / (nu rho) - B a~ and
// w_{j+1} = z / rho - B g~ - (q_j.z / rho) q_j (a~ = a / rho, g~ = g / rho;
// one pass over the basis, two updates per loaded value); q_j goes to the
// basis, w_{j+1} to the other work vector, nu_{j+1} = ||w_{j+1}||.
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_lz_d3(LzArgs<V> a, int j, double breakdown) {
  __shared__ double sm[RSB_WARPS];
  __shared__ V ca[RSB_MAXC], cg[RSB_MAXC];
  __shared__ double out[1];
  const Tile t = a.tiles[blockIdx.x];
  Unit& u = a.units[t.unit];
  if (u.status != U_ACTIVE || j >= u.msteps || j < u.j0) return;
  const int nd = u.nd;
  const int nb = 1 + nd + j;
  stage_coef<V, false>(u.c2, nb, u.isn, ca);
  stage_coef<V, false>(u.c1, nb, u.isn, cg);
  const V ssrc = V(u.dz_src), sz = V(u.dz_z), sqz = V(u.dz_qz);
  const V* src = (j & 1) ? a.W1 : a.W0;
  V* dst = (j & 1) ? a.W0 : a.W1;
  const V* z = a.AP;
  V* qj = a.Q + (long long)j * a.N;
  Acc<V> acc;
  unsigned long long pbytes = 0;
  for (int base = t.row0; base < t.row1; base += SUBROWS) {
    const int end = min(t.row1, base + SUBROWS);
    V q[RSB_SUBR], w[RSB_SUBR];
    bool ok[RSB_SUBR];
#pragma unroll
    for (int rr = 0; rr < RSB_SUBR; ++rr) {
      const int r = base + rr * RSB_BLOCK + threadIdx.x;
      ok[rr] = r < end;
      q[rr] = ok[rr] ? ssrc * src[r] : V(0);
      w[rr] = ok[rr] ? sz * z[r] : V(0);
      if (ok[rr] && unit_has(u, a.ckey, r)) {
        q[rr] -= ca[0];
        w[rr] -= cg[0];
      }
    }
    for (int l = 0; l < nd; ++l) {
      const double* d = l == 0 ? a.D0 : a.D1;
#pragma unroll
      for (int rr = 0; rr < RSB_SUBR; ++rr) {
        const int r = base + rr * RSB_BLOCK + threadIdx.x;
        if (ok[rr]) {
          const V dv = V(d[r]);
          q[rr] -= ca[1 + l] * dv;
          w[rr] -= cg[1 + l] * dv;
        }
      }
    }
    const V* cqa = ca + 1 + nd;
    const V* cqg = cg + 1 + nd;
    int k = 0;
    for (; k + 4 <= j; k += 4) {  // four basis vectors per round
      V qv[4][RSB_SUBR];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const V* qk = a.Q + (long long)(k + i) * a.N + base + threadIdx.x;
#pragma unroll
        for (int rr = 0; rr < RSB_SUBR; ++rr) qv[i][rr] = ok[rr] ? qk[rr * RSB_BLOCK] : V(0);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const V ka = cqa[k + i], kg = cqg[k + i];
#pragma unroll
        for (int rr = 0; rr < RSB_SUBR; ++rr) {
          q[rr] -= ka * qv[i][rr];
          w[rr] -= kg * qv[i][rr];
        }
      }
    }
    for (; k < j; ++k) {
      const V ka = cqa[k], kg = cqg[k];
      const V* qk = a.Q + (long long)k * a.N + base + threadIdx.x;
#pragma unroll
      for (int rr = 0; rr < RSB_SUBR; ++rr)
        if (ok[rr]) {
          const V b = qk[rr * RSB_BLOCK];
          q[rr] -= ka * b;
          w[rr] -= kg * b;
        }
    }
#pragma unroll
    for (int rr = 0; rr < RSB_SUBR; ++rr) {
      const int r = base + rr * RSB_BLOCK + threadIdx.x;
      if (ok[rr]) {
        w[rr] -= sqz * q[rr];
        qj[r] = q[rr];
        dst[r] = w[rr];
        acc.add(w[rr] * w[rr]);
        if (a.pb_b) pbytes += sizeof(V) * (unsigned long long)(4 + j) + 8ull * nd;
      }
    }
  }
  if (a.pb_b) prof_add(a.pb_b, pbytes);
  const double sum = block_total(acc, sm);
  if (threadIdx.x == 0) a.partials[blockIdx.x] = sum;
  if (last_cta(&u.cnt, u.ntile)) {
    final_reduce(a.partials, a.stride, u.tile0, u.ntile, 1, out);
    if (threadIdx.x == 0) {
      const double b = sqrt(out[0]);
      u.beta[j + 1] = b;
      if (b <= breakdown * u.dmax) {  // invariant subspace: the cycle ends here
        u.msteps = j + 1;
        u.broke = 1;
      }
    }
  }
}

// ----------------------------------------------------------------------------
// Ritz pairs of S (K x K, K <= 40): parallel cyclic Jacobi in one CTA (FP64).
// Rounds of the round-robin ("circle") ordering rotate K/2 disjoint pairs at
// once; each rotation is the symmetric 2x2 Schur rotation (Golub & Van Loan
// §8.5).  Output: theta_0..theta_kk (ascending) and their eigenvectors as the
// Y columns of the unit's storage.
// ----------------------------------------------------------------------------
template <typename T>
struct JacShared {
  T A[RSB_MAXM][RSB_MAXM + 1];
  T Z[RSB_MAXM][RSB_MAXM + 1];
  T c[RSB_MAXM / 2], s[RSB_MAXM / 2];
  int p[RSB_MAXM / 2], q[RSB_MAXM / 2];
  double red[RSB_WARPS];
  int rank[RSB_MAXM];
};

// T = double for the FP64 path; T = float for the mixed path, whose Lanczos
// vectors are FP32 (so FP32-accurate Ritz vectors lose nothing) and whose
// eigenvalue comes from the FP64 Rayleigh quotient at the end.
// Rotation (c, s) of the symmetric 2x2 Schur step for (a_pp, a_qq, a_pq)
// (Golub & Van Loan 8.5): t = sign(tau) / (|tau| + sqrt(1 + tau^2)) with
// tau = (a_qq - a_pp) / (2 a_pq), c = 1 / sqrt(1 + t^2), s = t c.  The angle t
// is taken in FP32 with fast division; c is normalised by Newton steps for
// 1 / sqrt(x) (c <- c (3 - x c^2) / 2) in the working precision, so that
// c^2 + s^2 = 1 to that precision.  Any t gives an orthogonal rotation; an
// FP32-accurate t leaves a_pq at ~1e-7 of its size instead of zero, which the
// following sweeps remove.  In FP64 this replaces two divisions and two square
// roots, long dependent chains on GB300's FP64 pipe.
// (an a_pq below FP32's range gives a non-finite angle: no rotation, t = 0)
__device__ __forceinline__ float jac_tan(float app, float aqq, float apq) {
  const float tau = __fdividef(aqq - app, 2.f * apq);
  const float t = __fdividef(copysignf(1.f, tau), fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f)));
  return isfinite(t) ? t : 0.f;
}
__device__ __forceinline__ void jac_rotation(float app, float aqq, float apq, float& c, float& s) {
  const float t = jac_tan(app, aqq, apq);
  const float x = fmaf(t, t, 1.f);
  float r = rsqrtf(x);
  r = r * fmaf(-0.5f * x, r * r, 1.5f);
  c = r;
  s = t * r;
}
__device__ __forceinline__ void jac_rotation(double app, double aqq, double apq, double& c,
                                             double& s) {
  const double t = (double)jac_tan(0.f, (float)(aqq - app), (float)apq);
  const double x = fma(t, t, 1.0);
  double r = (double)rsqrtf((float)x);
  r = r * fma(-0.5 * x, r * r, 1.5);
  r = r * fma(-0.5 * x, r * r, 1.5);
  c = r;
  s = t * r;
}

// tasks per thread and round: np*np + np*n2 <= 20*20 + 20*40 over RSB_BLOCK threads
#define EIG_TASKS ((RSB_MAXM * RSB_MAXM * 3 / 4 + RSB_BLOCK - 1) / RSB_BLOCK)

template <typename T, bool CO>
__device__ void lz_eig_u(Unit& u, double* Sm, JacShared<T>& J) {
  if (ldc<CO>(&u.status) != U_ACTIVE) return;
  const int tid = threadIdx.x;
  const int K = ldc<CO>(&u.msteps);
  const int n2 = K + (K & 1);
  for (int idx = tid; idx < n2 * n2; idx += RSB_BLOCK) {
    const int i = idx / n2, k = idx % n2;
    J.A[i][k] = (i < K && k < K) ? T(ldc<CO>(Sm + i * RSB_MAXM + k)) : T(0);
    J.Z[i][k] = i == k ? T(1) : T(0);
  }
  __syncthreads();
  double fro = 0.0;
  for (int idx = tid; idx < K * K; idx += RSB_BLOCK) {
    const double x = (double)J.A[idx / K][idx % K];
    fro += x * x;
  }
  fro = block_sum(fro, J.red);
  if (tid == 0) J.red[0] = fro;
  __syncthreads();
  fro = J.red[0];
  __syncthreads();
  const double eps2 = sizeof(T) == 8 ? 1e-30 : 1e-14;
  const double thr = fro * eps2;
  // this thread's tasks of every round: np*np blocks of A (pair i1 x pair i2),
  // then np*n2 (pair, row) updates of Z; fixed for the whole solve
  const int np = n2 / 2;
  int ta[EIG_TASKS], tb[EIG_TASKS];
#pragma unroll
  for (int k = 0; k < EIG_TASKS; ++k) {
    const int task = tid + k * RSB_BLOCK;
    ta[k] = -1;
    tb[k] = 0;
    if (task < np * np) {
      ta[k] = task / np;
      tb[k] = task - ta[k] * np;
    } else if (task < np * np + np * n2) {
      const int zt = task - np * np;
      ta[k] = -2;
      tb[k] = ((zt / n2) << 8) | (zt % n2);
    }
  }
  for (int sweep = 0; sweep < 20; ++sweep) {
    double off = 0.0;
    for (int idx = tid; idx < K * K; idx += RSB_BLOCK) {
      const int i = idx / K, k = idx % K;
      if (i < k) off += (double)J.A[i][k] * (double)J.A[i][k];
    }
    off = block_sum(off, J.red);
    if (tid == 0) J.red[0] = off;
    __syncthreads();
    off = J.red[0];
    __syncthreads();
    if (off <= thr) break;
    for (int rnd = 0; rnd < n2 - 1; ++rnd) {
      if (tid < np) {
        // round-robin pairing: slot 0 holds index 0, the others rotate
        int ia = tid + rnd - 1, ib = n2 - 2 - tid + rnd;
        if (ia >= n2 - 1) ia -= n2 - 1;
        if (ib >= n2 - 1) ib -= n2 - 1;
        int pa = tid == 0 ? 0 : ia + 1;
        int pb = ib + 1;
        if (pa > pb) { const int tt = pa; pa = pb; pb = tt; }
        T cc = T(1), ss = T(0);
        const T apq = J.A[pa][pb];
        if (pb < K && apq != T(0)) jac_rotation(J.A[pa][pa], J.A[pb][pb], apq, cc, ss);
        J.p[tid] = pa;
        J.q[tid] = pb;
        J.c[tid] = cc;
        J.s[tid] = ss;
      }
      __syncthreads();
      // the round's rotations act on disjoint index pairs, so every 2x2 block
      // (pair i1 rows, pair i2 columns) is updated in place by one thread:
      // the column rotation, then the row rotation; Z takes the column one
#pragma unroll
      for (int k = 0; k < EIG_TASKS; ++k) {
        if (ta[k] >= 0) {
          const int i1 = ta[k], i2 = tb[k];
          const int p1 = J.p[i1], q1 = J.q[i1], p2 = J.p[i2], q2 = J.q[i2];
          const T c1 = J.c[i1], s1 = J.s[i1], c2 = J.c[i2], s2 = J.s[i2];
          const T a11 = J.A[p1][p2], a12 = J.A[p1][q2], a21 = J.A[q1][p2], a22 = J.A[q1][q2];
          const T b11 = c2 * a11 - s2 * a12, b12 = s2 * a11 + c2 * a12;
          const T b21 = c2 * a21 - s2 * a22, b22 = s2 * a21 + c2 * a22;
          J.A[p1][p2] = c1 * b11 - s1 * b21;
          J.A[q1][p2] = s1 * b11 + c1 * b21;
          J.A[p1][q2] = c1 * b12 - s1 * b22;
          J.A[q1][q2] = s1 * b12 + c1 * b22;
        } else if (ta[k] == -2) {
          const int i = tb[k] >> 8, r = tb[k] & 255;
          const int pa = J.p[i], pb = J.q[i];
          const T cc = J.c[i], ss = J.s[i];
          const T zx = J.Z[r][pa], zy = J.Z[r][pb];
          J.Z[r][pa] = cc * zx - ss * zy;
          J.Z[r][pb] = ss * zx + cc * zy;
        }
      }
      __syncthreads();
    }
  }
  // ascending order (ties by index)
  if (tid < K) {
    const T e = J.A[tid][tid];
    int rk = 0;
    for (int l = 0; l < K; ++l) {
      const T f = J.A[l][l];
      rk += (f < e) || (f == e && l < tid);
    }
    J.rank[tid] = rk;
  }
  __syncthreads();
  const int kk = ldc<CO>(&u.broke) ? 0 : min(u.keep, K - 1);
  double* Ym = Sm + RSB_MAXM * RSB_MAXM;
  for (int idx = tid; idx < K * K; idx += RSB_BLOCK) {
    const int l = idx / K, i = idx % K;  // eigenvector i (unsorted), component l
    const int rk = J.rank[i];
    if (rk <= kk) Ym[l * RSB_MAXM + rk] = (double)J.Z[l][i];
  }
  if (tid < K) {
    const int rk = J.rank[tid];
    if (rk <= kk) u.th[rk] = (double)J.A[tid][tid];
    if (rk == 0) u.theta = (double)J.A[tid][tid];
  }
  if (tid == 0) u.kk = kk;
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(RSB_BLOCK) k_lz_eig(Unit* units, double* S, int nunits) {
  __shared__ JacShared<T> J;
  if ((int)blockIdx.x >= nunits) return;
  lz_eig_u<T, false>(units[blockIdx.x], unit_S(S, blockIdx.x), J);
}

// The Ritz-pair launch for other solvers of the library (block Lanczos).
int launch_lz_eig(int f32, Unit* units, double* S, int nunits, cudaStream_t s) {
  if (f32) k_lz_eig<float><<<nunits, RSB_BLOCK, 0, s>>>(units, S, nunits);
  else k_lz_eig<double><<<nunits, RSB_BLOCK, 0, s>>>(units, S, nunits);
  RSB_CKL("k_lz_eig");
  return RSB_OK;
}

// ----------------------------------------------------------------------------
// Ritz vector and thick-restart basis (per row, in place): y = Q s_0 into Y;
// q_i <- Q s_i for i < kk; the residual direction moves to W[kk & 1] so that
// the next cycle's first step reads it.
// ----------------------------------------------------------------------------
template <typename V, bool CO>
__device__ __forceinline__ void lz_ritz_t(const LzArgs<V>& a, int tix) {
  const Tile t = a.tiles[tix];
  const Unit& u = a.units[t.unit];
  if (ldc<CO>(&u.status) != U_ACTIVE) return;
  const int K = ldc<CO>(&u.msteps);
  const int kk = ldc<CO>(&u.kk);
  const double* Ym = unit_S(a.S, t.unit) + RSB_MAXM * RSB_MAXM;
  const V* wl = (K & 1) ? a.W1 : a.W0;
  V* wn = (kk & 1) ? a.W1 : a.W0;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    V q[RSB_MAXM];
#pragma unroll
    for (int l = 0; l < RSB_MAXM; ++l) q[l] = l < K ? a.Q[(long long)l * a.N + r] : V(0);
    for (int i = 0; i <= kk; ++i) {
      V acc = V(0);
#pragma unroll
      for (int l = 0; l < RSB_MAXM; ++l)
        if (l < K) acc += V(ldc<CO>(Ym + l * RSB_MAXM + i)) * q[l];
      if (i == 0) a.Y[r] = acc;
      if (i < kk) a.Q[(long long)i * a.N + r] = acc;
    }
    if (kk > 0 && wn != wl) wn[r] = wl[r];
  }
  if (CO && a.pb_a && threadIdx.x == 0)
    atomicAdd(a.pb_a, (unsigned long long)(t.row1 - t.row0) * sizeof(V) * (K + kk + 1));
}

// Residual of y with theta, plus the projection dots of y against the fixed
// basis.  mode 0: Lanczos cycle end (decides convergence); mode 1: the start
// vector only (no residual).
template <typename V, bool CO>
__device__ __forceinline__ void lz_resid_t(const LzArgs<V>& a, const V* y, int mode, int tix,
                                           double* sm, double* out) {
  const Tile t = a.tiles[tix];
  Unit& u = a.units[t.unit];
  if (ldc<CO>(&u.status) != U_ACTIVE) return;
  const int nd = u.nd;
  const V th = V(ldc<CO>(&u.theta));
  Acc<V> r2, y2, ys, d0, d1;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    const V yr = y[r];
    if (mode == 0) {
      const V res = spmv_row<V, CO>(a.slice_ptr, a.ent, y, r, yr) - th * yr;
      r2.add(res * res);
    }
    y2.add(yr * yr);
    ys.add(yr);
    if (nd > 0) d0.add(V(a.D0[r]) * yr);
    if (nd > 1) d1.add(V(a.D1[r]) * yr);
  }
  if (CO && a.pb_a && threadIdx.x == 0) {
    unsigned long long b = 0;
    for (int r = t.row0; r < t.row1; ++r) b += 4ull * row_width(a.slice_ptr, r);
    b += (unsigned long long)(t.row1 - t.row0) * (sizeof(V) + 8ull * nd);
    atomicAdd(a.pb_a, b);
  }
  double v[5] = {r2.get(), y2.get(), ys.get(), d0.get(), d1.get()};
  const int nv = 3 + nd;
  for (int c = 0; c < nv; ++c) {
    const double sum = block_sum(v[c], sm);
    if (threadIdx.x == 0) a.partials[(long long)c * a.stride + tix] = sum;
  }
  if (last_cta(&u.cnt, u.ntile)) {
    final_reduce(a.partials, a.stride, u.tile0, u.ntile, nv, out);
    if (threadIdx.x == 0) {
      u.ynorm2 = out[1];
      u.cp[0] = out[2] * u.isn;
      for (int l = 0; l < nd; ++l) u.cp[1 + l] = out[3 + l];
      if (mode == 0) {
        u.resid = sqrt(out[0] / out[1]);
        u.cycles += 1;
        atomicAdd((unsigned long long*)a.stat_cycles, 1ull);
        int st = U_ACTIVE;
        if (u.resid <= u.tolabs) st = U_CONVERGED;
        else if (u.cycles >= u.maxcycles) st = U_CAPPED;
        if (st != U_ACTIVE) {
          u.status = st;
          atomicSub(a.n_active, 1);
        } else if (u.kk > 0) {
          // thick restart: the kept Ritz vectors occupy q_0..q_{kk-1}; the next
          // cycle starts at step kk from the residual direction
          u.beta0 = u.beta[u.msteps];
          u.j0 = u.kk;
          u.msteps = u.m;
          atomicMin(a.jmin, u.kk);
        } else {
          u.j0 = 0;  // explicit restart from y (proj2/proj3 follow)
          atomicMin(a.jmin, 0);
        }
      }
    }
    if (mode == 0) {
      __syncthreads();
      // next cycle's S = diag(kept Ritz values); explicit restarts clear it all
      if (u.status == U_ACTIVE) {
        double* Sm = unit_S(a.S, t.unit);
        const int kk = u.kk;
        for (int idx = threadIdx.x; idx < RSB_MAXM * RSB_MAXM; idx += RSB_BLOCK) {
          const int i = idx / RSB_MAXM, k = idx % RSB_MAXM;
          Sm[idx] = (i == k && i < kk) ? u.th[i] : 0.0;
        }
      }
    }
  }
}

// Explicit restart only (a cycle that ended on an invariant subspace without
// converging): y -= B cp (in place); dots of the result against B -> c2.
template <typename V, bool CO>
__device__ __forceinline__ void proj2_t(const LzArgs<V>& a, V* y, int tix, double* sm,
                                        double* out) {
  const Tile t = a.tiles[tix];
  Unit& u = a.units[t.unit];
  if (ldc<CO>(&u.status) != U_ACTIVE || ldc<CO>(&u.j0) != 0) return;
  const int nd = u.nd;
  const double cp0 = ldc<CO>(&u.cp[0]), cp1 = ldc<CO>(&u.cp[1]), cp2 = ldc<CO>(&u.cp[2]);
  Acc<V> ys, d0, d1;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    V v = y[r];
    if (unit_has(u, a.ckey, r)) v -= V(cp0 * u.isn);
    if (nd > 0) v -= V(cp1) * V(a.D0[r]);
    if (nd > 1) v -= V(cp2) * V(a.D1[r]);
    y[r] = v;
    ys.add(v);
    if (nd > 0) d0.add(V(a.D0[r]) * v);
    if (nd > 1) d1.add(V(a.D1[r]) * v);
  }
  if (CO && a.pb_a && threadIdx.x == 0)
    atomicAdd(a.pb_a, (unsigned long long)(t.row1 - t.row0) * (2 * sizeof(V) + 8ull * nd));
  double v[3] = {ys.get(), d0.get(), d1.get()};
  const int nv = 1 + nd;
  for (int c = 0; c < nv; ++c) {
    const double sum = block_sum(v[c], sm);
    if (threadIdx.x == 0) a.partials[(long long)c * a.stride + tix] = sum;
  }
  if (last_cta(&u.cnt, u.ntile)) {
    final_reduce(a.partials, a.stride, u.tile0, u.ntile, nv, out);
    if (threadIdx.x == 0) {
      u.c2[0] = out[0] * u.isn;
      for (int l = 0; l < nd; ++l) u.c2[1 + l] = out[1 + l];
    }
  }
}

// w0 = y - B c2 (second pass), beta0 = ||w0||; a cycle starts at step 0.
template <typename V, bool CO>
__device__ __forceinline__ void proj3_t(const LzArgs<V>& a, const V* y, int tix, double* sm,
                                        double* out) {
  const Tile t = a.tiles[tix];
  Unit& u = a.units[t.unit];
  if (ldc<CO>(&u.status) != U_ACTIVE || ldc<CO>(&u.j0) != 0) return;
  const int nd = u.nd;
  const double c20 = ldc<CO>(&u.c2[0]), c21 = ldc<CO>(&u.c2[1]), c22 = ldc<CO>(&u.c2[2]);
  Acc<V> acc;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    V v = y[r];
    if (unit_has(u, a.ckey, r)) v -= V(c20 * u.isn);
    if (nd > 0) v -= V(c21) * V(a.D0[r]);
    if (nd > 1) v -= V(c22) * V(a.D1[r]);
    a.W0[r] = v;
    acc.add(v * v);
  }
  if (CO && a.pb_a && threadIdx.x == 0)
    atomicAdd(a.pb_a, (unsigned long long)(t.row1 - t.row0) * (2 * sizeof(V) + 8ull * nd));
  const double sum = block_sum(acc.get(), sm);
  if (threadIdx.x == 0) a.partials[tix] = sum;
  if (last_cta(&u.cnt, u.ntile)) {
    final_reduce(a.partials, a.stride, u.tile0, u.ntile, 1, out);
    if (threadIdx.x == 0) {
      u.beta0 = sqrt(out[0]);
      u.msteps = u.m;
      u.broke = 0;
    }
  }
}

template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_lz_ritz(LzArgs<V> a) {
  lz_ritz_t<V, false>(a, blockIdx.x);
}
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_lz_resid(LzArgs<V> a, const V* __restrict__ y,
                                                        int mode) {
  __shared__ double sm[RSB_WARPS];
  __shared__ double out[3 + RSB_MAXD];
  lz_resid_t<V, false>(a, y, mode, blockIdx.x, sm, out);
}
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_proj2(LzArgs<V> a, V* __restrict__ y) {
  __shared__ double sm[RSB_WARPS];
  __shared__ double out[1 + RSB_MAXD];
  proj2_t<V, false>(a, y, blockIdx.x, sm, out);
}
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_proj3(LzArgs<V> a, const V* __restrict__ y) {
  __shared__ double sm[RSB_WARPS];
  __shared__ double out[1];
  proj3_t<V, false>(a, y, blockIdx.x, sm, out);
}

// ----------------------------------------------------------------------------
// Persistent cooperative kernel: one whole Lanczos cycle (steps j0..M-1, the
// Ritz pairs of S, Ritz vector and restart basis, residual) in one launch.
// CTAs walk the tiles grid-stride (the same CTA owns the same tiles in every
// phase); phases are separated by the bounded grid barrier; reductions keep
// the last-CTA scheme, whose result the barrier publishes.
// ----------------------------------------------------------------------------
template <typename V>
union CycleShared {
  JacShared<V> J;
  double wsd[SUBROWS];
};

template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK, 2)
    k_lz_cycle(LzArgs<V> a, int jstart, int M, double breakdown, int ntiles, int nunits,
               GridBar* gb) {
  __shared__ CycleShared<V> sh;
  __shared__ double out[RSB_MAXC];
  __shared__ double sm[RSB_WARPS];
  __shared__ V cv[RSB_MAXC];
  V* ws = reinterpret_cast<V*>(sh.wsd);
  const unsigned G = gridDim.x;
  for (int j = jstart; j < M; ++j) {
    for (int t = blockIdx.x; t < ntiles; t += G) lz_a_t<V, true>(a, j, t, ws, out);
    if (!grid_sync(gb, G)) return;
    for (int t = blockIdx.x; t < ntiles; t += G) lz_b_t<V, true>(a, j, t, ws, cv, out);
    if (!grid_sync(gb, G)) return;
    for (int t = blockIdx.x; t < ntiles; t += G) lz_c_t<V, true>(a, j, breakdown, t, cv, sm, out);
    if (!grid_sync(gb, G)) return;
  }
  for (int u = blockIdx.x; u < nunits; u += G) lz_eig_u<V, true>(a.units[u], unit_S(a.S, u), sh.J);
  if (!grid_sync(gb, G)) return;
  for (int t = blockIdx.x; t < ntiles; t += G) lz_ritz_t<V, true>(a, t);
  if (!grid_sync(gb, G)) return;
  for (int t = blockIdx.x; t < ntiles; t += G) lz_resid_t<V, true>(a, a.Y, 0, t, sm, out);
  if (!grid_sync(gb, G)) return;
  for (int t = blockIdx.x; t < ntiles; t += G) proj2_t<V, true>(a, a.Y, t, sm, out);
  if (!grid_sync(gb, G)) return;
  for (int t = blockIdx.x; t < ntiles; t += G) proj3_t<V, true>(a, a.Y, t, sm, out);
}

// ----------------------------------------------------------------------------
// Resident persistent solve (launch mode 3).  When every tile of the level can
// own one co-resident CTA and the tile's rows of the basis fit in that CTA's
// shared memory (the level's basis is at most the chip's shared memory: the
// 131,072-row level with 40 FP32 vectors is 21 MB over 256 CTAs), one
// cooperative launch runs every cycle of the solve.  The Gram-Schmidt passes
// then read q_0..q_j from shared memory; global memory carries the SpMV
// operand, the reduction partials and the per-unit scalars.  Steps, their
// order, the per-thread accumulation order and the reductions are those of
// the streaming kernels above, so both modes give the same numbers.
// Shared layout: JacShared | coefficients (FP64, and in the vector type) | w
// (z) of the tile | v of the tile (FP32) | deflation vectors of the tile |
// Q[k * trs + rl].
// ----------------------------------------------------------------------------
__host__ __device__ constexpr size_t res_align(size_t b) { return (b + 15) & ~(size_t)15; }

template <typename V>
__host__ __device__ constexpr size_t res_smem_bytes(int M, int trs) {
  return res_align(sizeof(JacShared<V>)) + res_align(2 * sizeof(double) * RSB_MAXC) +
         res_align(2 * sizeof(V) * RSB_MAXC) + 2 * res_align(sizeof(V) * (size_t)trs) +
         res_align(sizeof(V) * RSB_MAXD * (size_t)trs) + sizeof(V) * (size_t)M * (size_t)trs;
}

// Dots of [1, D, q_0..] with the tile's w: the coefficient split across warps
// and the per-lane row order of tile_dots.
template <typename V>
__device__ __forceinline__ void res_dots(const Tile& t, int nd, int nc, const V* Qs,
                                         const V* Ds, int trs, const V* ws,
                                         Acc<V> (&acc)[MAXCW]) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nr = t.row1 - t.row0;
#pragma unroll
  for (int i = 0; i < MAXCW; ++i) {
    const int c = w + RSB_WARPS * i;
    if (c < nc) {
      if (c == 0) {
        for (int rl = lane; rl < nr; rl += 32) acc[i].add(V(1) * ws[rl]);
      } else if (c <= nd) {
        const V* d = Ds + (size_t)(c - 1) * trs;
        for (int rl = lane; rl < nr; rl += 32) acc[i].add(d[rl] * ws[rl]);
      } else {
        const V* q = Qs + (size_t)(c - 1 - nd) * trs;
        for (int rl = lane; rl < nr; rl += 32) acc[i].add(q[rl] * ws[rl]);
      }
    }
  }
}

// w -= [1/sqrt(n), D, q_0..q_{nq-1}] cv, in the order of gs_update_rows (cv:
// the coefficients in the vector type; in_unit: the row belongs to the unit).
template <typename V>
__device__ __forceinline__ V res_upd_row(const V* cv, int nd, int nq, const V* Qs,
                                         const V* Ds, int trs, int rl, bool in_unit, V w) {
  if (in_unit) w -= cv[0];
  for (int l = 0; l < nd; ++l) w -= cv[1 + l] * Ds[(size_t)l * trs + rl];
  const V* cq = cv + 1 + nd;
  for (int k = 0; k < nq; ++k) w -= cq[k] * Qs[(size_t)k * trs + rl];
  return w;
}

template <typename V>
__device__ __forceinline__ void res_store_dots(double* P, long long stride, int nc,
                                               Acc<V> (&acc)[MAXCW], int tix) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < MAXCW; ++i) {
    const int c = w + RSB_WARPS * i;
    if (c < nc) {
      const double s = warp_total(acc[i]);
      if (lane == 0) P[(long long)c * stride + tix] = s;
    }
  }
}

// The step phases write per-tile partials into P; after the grid barrier
// every CTA of the unit reduces them itself (fixed order, so all CTAs hold
// the same coefficients), which takes the last-CTA ticket and the staging of
// the coefficients off the critical path.  Consecutive phases alternate
// between two partial buffers: a buffer is rewritten only after a barrier
// that follows every CTA's reduction of its previous contents.
//
// A(j): q_j = src * s into shared memory, w = L q_j, dots [1, D, q_0..q_j]^T w.
template <typename V>
__device__ void res_a(const LzArgs<V>& a, int j, V s, int tix, const Tile& t, const Unit& u,
                      V* Qs, const V* Ds, int trs, V* ws, double* P) {
  const int nr = t.row1 - t.row0;
  const V* src = (j & 1) ? a.W1 : a.W0;
  const int nd = u.nd;
  const int nc = 2 + nd + j;
  unsigned long long pbytes = 0;
  for (int rl = threadIdx.x; rl < nr; rl += RSB_BLOCK) {
    const int r = t.row0 + rl;
    const V xr = __ldcg(src + r);
    ws[rl] = s * spmv_row<V, true>(a.slice_ptr, a.ent, src, r, xr);
    Qs[(size_t)j * trs + rl] = s * xr;
    if (a.pb_a)
      pbytes += 4ull * row_width(a.slice_ptr, r) + sizeof(V) * (unsigned long long)(4 + j) +
                8ull * nd;
  }
  __syncthreads();
  Acc<V> acc[MAXCW];
  res_dots<V>(t, nd, nc, Qs, Ds, trs, ws, acc);
  res_store_dots<V>(P, a.stride, nc, acc, tix);
  if (a.pb_a) prof_add(a.pb_a, pbytes);
}

// B(j): w -= basis c1, dots of the result (second pass).
template <typename V>
__device__ void res_b(const LzArgs<V>& a, int j, int tix, const Tile& t, int nd, bool masked,
                      uint64_t key, const V* Qs, const V* Ds, int trs, V* ws, const V* cv,
                      double* P) {
  const int nr = t.row1 - t.row0;
  const int nc = 2 + nd + j;
  unsigned long long pbytes = 0;
  for (int rl = threadIdx.x; rl < nr; rl += RSB_BLOCK) {
    const bool in_unit = !masked || a.ckey[t.row0 + rl] == key;
    ws[rl] = res_upd_row<V>(cv, nd, j + 1, Qs, Ds, trs, rl, in_unit, ws[rl]);
    if (a.pb_b) pbytes += sizeof(V) * (unsigned long long)(3 + j) + 8ull * nd;
  }
  __syncthreads();
  Acc<V> acc[MAXCW];
  res_dots<V>(t, nd, nc, Qs, Ds, trs, ws, acc);
  res_store_dots<V>(P, a.stride, nc, acc, tix);
  if (a.pb_b) prof_add(a.pb_b, pbytes);
}

// C(j): w -= basis c2 into W[(j + 1) & 1] (the next SpMV operand), ||w||^2.
template <typename V>
__device__ void res_c(const LzArgs<V>& a, int j, int tix, const Tile& t, int nd, bool masked,
                      uint64_t key, const V* Qs, const V* Ds, int trs, const V* ws,
                      const V* cv, double* sm, double* P) {
  const int nr = t.row1 - t.row0;
  V* dst = (j & 1) ? a.W0 : a.W1;
  Acc<V> acc;
  unsigned long long pbytes = 0;
  for (int rl = threadIdx.x; rl < nr; rl += RSB_BLOCK) {
    const bool in_unit = !masked || a.ckey[t.row0 + rl] == key;
    const V w = res_upd_row<V>(cv, nd, j + 1, Qs, Ds, trs, rl, in_unit, ws[rl]);
    dst[t.row0 + rl] = w;
    acc.add(w * w);
    if (a.pb_c) pbytes += sizeof(V) * (unsigned long long)(3 + j) + 8ull * nd;
  }
  if (a.pb_c) prof_add(a.pb_c, pbytes);
  const double sum = block_total(acc, sm);
  if (threadIdx.x == 0) P[tix] = sum;
}

// FP32 steps with the delayed second pass (D1-D3 of the streaming kernels,
// in their order).  D1(j): v = src rows into vs, z = L (src / nu) into ws.
template <typename V>
__device__ void res_d1(const LzArgs<V>& a, int j, V s, const Tile& t, V* vs, V* ws) {
  const int nr = t.row1 - t.row0;
  const V* src = (j & 1) ? a.W1 : a.W0;
  unsigned long long pbytes = 0;
  for (int rl = threadIdx.x; rl < nr; rl += RSB_BLOCK) {
    const int r = t.row0 + rl;
    const V xr = __ldcg(src + r);
    vs[rl] = xr;
    ws[rl] = s * spmv_row<V, true>(a.slice_ptr, a.ent, src, r, xr);
    if (a.pb_a) pbytes += 4ull * row_width(a.slice_ptr, r) + 2ull * sizeof(V);
  }
  if (a.pb_a) prof_add(a.pb_a, pbytes);
  __syncthreads();
}

// D2(j): dots of v (vs) and z (ws) with [1, D, q_0..q_{j-1}] and with v, in the
// per-lane order of k_lz_d2 (partials [a_b, v.v] then [g_b, v.z]).
template <typename V>
__device__ void res_d2(const LzArgs<V>& a, int j, int tix, const Tile& t, int nd, const V* Qs,
                       const V* Ds, int trs, const V* vs, const V* ws, double* P) {
  const int nr = t.row1 - t.row0;
  const int nb = 1 + nd + j;
  const int nc = nb + 1;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Acc<V> av[MAXCW], az[MAXCW];
#pragma unroll
  for (int i = 0; i < MAXCW; ++i) {
    const int c = w + RSB_WARPS * i;
    if (c < nc) {
      if (c == 0) {
        for (int rl = lane; rl < nr; rl += 32) {
          av[i].add(vs[rl]);
          az[i].add(ws[rl]);
        }
      } else if (c <= nd) {
        const V* d = Ds + (size_t)(c - 1) * trs;
        for (int rl = lane; rl < nr; rl += 32) {
          av[i].add(d[rl] * vs[rl]);
          az[i].add(d[rl] * ws[rl]);
        }
      } else {
        const V* q = c < nb ? Qs + (size_t)(c - 1 - nd) * trs : vs;
        for (int rl = lane; rl < nr; rl += 32) {
          const V qv = q[rl];
          av[i].add(qv * vs[rl]);
          az[i].add(qv * ws[rl]);
        }
      }
    }
  }
  res_store_dots<V>(P, a.stride, nc, av, tix);
  res_store_dots<V>(P + (long long)nc * a.stride, a.stride, nc, az, tix);
  if (a.pb_a2) {
    unsigned long long pbytes = 0;
    for (int rl = threadIdx.x; rl < nr; rl += RSB_BLOCK)
      pbytes += sizeof(V) * (unsigned long long)(2 + j) + 8ull * nd;
    prof_add(a.pb_a2, pbytes);
  }
}

// D3(j): q_j = ssrc v - B ca into Qs, w = sz z - B cg - sqz q_j into
// W[(j + 1) & 1], ||w||^2 (the per-row order of k_lz_d3).
template <typename V>
__device__ void res_d3(const LzArgs<V>& a, int j, int tix, const Tile& t, int nd, bool masked,
                       uint64_t key, V* Qs, const V* Ds, int trs, const V* vs, const V* ws,
                       const V* ca, const V* cg, V ssrc, V sz, V sqz, double* sm, double* P) {
  const int nr = t.row1 - t.row0;
  V* dst = (j & 1) ? a.W0 : a.W1;
  Acc<V> acc;
  unsigned long long pbytes = 0;
  for (int rl = threadIdx.x; rl < nr; rl += RSB_BLOCK) {
    const bool in_unit = !masked || a.ckey[t.row0 + rl] == key;
    V q = ssrc * vs[rl];
    V w = sz * ws[rl];
    if (in_unit) {
      q -= ca[0];
      w -= cg[0];
    }
    for (int l = 0; l < nd; ++l) {
      const V dv = Ds[(size_t)l * trs + rl];
      q -= ca[1 + l] * dv;
      w -= cg[1 + l] * dv;
    }
    for (int k = 0; k < j; ++k) {
      const V b = Qs[(size_t)k * trs + rl];
      q -= ca[1 + nd + k] * b;
      w -= cg[1 + nd + k] * b;
    }
    w -= sqz * q;
    Qs[(size_t)j * trs + rl] = q;
    dst[t.row0 + rl] = w;
    acc.add(w * w);
    if (a.pb_b) pbytes += sizeof(V) * (unsigned long long)(4 + j) + 8ull * nd;
  }
  if (a.pb_b) prof_add(a.pb_b, pbytes);
  const double sum = block_total(acc, sm);
  if (threadIdx.x == 0) P[tix] = sum;
}

// coefficients of a finished reduction: c[0] carries the 1/sqrt(n) of u0 (as
// the streaming kernels store it); cv the same in the vector type, cv[0]
// already times 1/sqrt(n) again (the u0 component of the update)
template <typename V>
__device__ __forceinline__ void res_coef(const double* out, int nc, double isn, double* c,
                                         V* cv) {
  for (int k = threadIdx.x; k < nc; k += RSB_BLOCK) {
    const double v = k == 0 ? out[0] * isn : out[k];
    c[k] = v;
    cv[k] = k == 0 ? V(v * isn) : V(v);
  }
  __syncthreads();
}

// Ritz vector y = Q s_0 into Y and the kept vectors q_i <- Q s_i (i < kk) in
// shared memory; the residual direction moves to W[kk & 1].
template <typename V>
__device__ void res_ritz(const LzArgs<V>& a, const Tile& t, const Unit& u, V* Qs, int trs,
                         V* Ys) {
  if (ldc<true>(&u.status) != U_ACTIVE) return;
  const int nr = t.row1 - t.row0;
  const int K = ldc<true>(&u.msteps);
  const int kk = ldc<true>(&u.kk);
  const double* Ym = unit_S(a.S, t.unit) + RSB_MAXM * RSB_MAXM;
  constexpr int YS = RSB_MAXKEEP + 1;
  for (int idx = threadIdx.x; idx < K * (kk + 1); idx += RSB_BLOCK) {
    const int l = idx / (kk + 1), i = idx % (kk + 1);
    Ys[l * YS + i] = V(__ldcg(Ym + l * RSB_MAXM + i));
  }
  __syncthreads();
  const V* wl = (K & 1) ? a.W1 : a.W0;
  V* wn = (kk & 1) ? a.W1 : a.W0;
  for (int rl = threadIdx.x; rl < nr; rl += RSB_BLOCK) {
    const int r = t.row0 + rl;
    V q[RSB_MAXM];
#pragma unroll
    for (int l = 0; l < RSB_MAXM; ++l) q[l] = l < K ? Qs[(size_t)l * trs + rl] : V(0);
    for (int i = 0; i <= kk; ++i) {
      V acc = V(0);
#pragma unroll
      for (int l = 0; l < RSB_MAXM; ++l)
        if (l < K) acc += Ys[l * YS + i] * q[l];
      if (i == 0) a.Y[r] = acc;
      if (i < kk) Qs[(size_t)i * trs + rl] = acc;
    }
    if (kk > 0 && wn != wl) wn[r] = __ldcg(wl + r);
  }
  if (a.pb_a && threadIdx.x == 0)
    atomicAdd(a.pb_a, (unsigned long long)nr * sizeof(V) * (K + kk + 1));
}

template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK, 2)
    k_lz_res(LzArgs<V> a, int M, int trs, double breakdown, int nunits, int maxcyc, GridBar* gb) {
  extern __shared__ __align__(16) unsigned char res_sh[];
  JacShared<V>& J = *reinterpret_cast<JacShared<V>*>(res_sh);
  size_t off = res_align(sizeof(JacShared<V>));
  double* c1 = reinterpret_cast<double*>(res_sh + off);
  double* c2 = c1 + RSB_MAXC;
  off += res_align(2 * sizeof(double) * RSB_MAXC);
  V* cv1 = reinterpret_cast<V*>(res_sh + off);
  V* cv2 = cv1 + RSB_MAXC;
  off += res_align(2 * sizeof(V) * RSB_MAXC);
  V* ws = reinterpret_cast<V*>(res_sh + off);
  off += res_align(sizeof(V) * (size_t)trs);
  V* vs = reinterpret_cast<V*>(res_sh + off);
  off += res_align(sizeof(V) * (size_t)trs);
  V* Ds = reinterpret_cast<V*>(res_sh + off);
  off += res_align(sizeof(V) * RSB_MAXD * (size_t)trs);
  V* Qs = reinterpret_cast<V*>(res_sh + off);
  __shared__ double out[2 * RSB_MAXC + 2];
  __shared__ double dsc[3], dsk[RSB_MAXM];
  __shared__ double sm[RSB_WARPS];
  __shared__ double beta_sh;
  __shared__ V scale_sh;
  const unsigned G = gridDim.x;
  const int tix = blockIdx.x;
  const Tile t = a.tiles[tix];
  Unit& u = a.units[t.unit];
  const int nr = t.row1 - t.row0;
  const int nd = u.nd;
  const bool masked = u.masked;
  const uint64_t key = u.key;
  const double isn = u.isn;
  const bool lead = tix == u.tile0 && threadIdx.x == 0;
  double* const Pb[2] = {a.partials, a.partials + (long long)RSB_MAXC * a.stride};
  // the tile's deflation vectors in the vector type, once per solve
  for (int l = 0; l < nd; ++l) {
    const double* d = l == 0 ? a.D0 : a.D1;
    for (int rl = threadIdx.x; rl < nr; rl += RSB_BLOCK) Ds[(size_t)l * trs + rl] = V(d[t.row0 + rl]);
  }
  __syncthreads();
  int* jm = a.jmin;  // two slots: read one at a cycle's start, refill the other
  for (int cyc = 0; cyc < maxcyc; ++cyc) {
    const int jstart = cyc == 0 ? 0 : min(max(__ldcg(jm + (cyc & 1)), 0), M);
    if (tix == 0 && threadIdx.x == 0) jm[(cyc + 1) & 1] = 0x7FFFFFFF;
    LzArgs<V> ac = a;
    ac.jmin = jm + ((cyc + 1) & 1);
    // the unit's step state, tracked identically by all of its CTAs
    const bool on = __ldcg(&u.status) == U_ACTIVE;
    const int j0 = __ldcg(&u.j0);
    int msteps = __ldcg(&u.msteps);
    if (threadIdx.x == 0) {
      beta_sh = __ldcg(&u.beta0);
      scale_sh = V(1.0 / beta_sh);
    }
    __syncthreads();
    int ph = 0;
    for (int j = jstart; j < M; ++j) {
      const bool st = on && j < msteps && j >= j0;
      if constexpr (sizeof(V) == 4) {
        // FP32: the streaming kernels' steps D1-D3 (second pass delayed);
        // partials: D2 in rows [0, 2 nc), the norm in row 2 RSB_MAXC, so that
        // no CTA rewrites rows another CTA of the unit may still reduce
        const int nb = 1 + nd + j;
        const int nc = nb + 1;
        double* Pn = a.partials + (long long)(2 * RSB_MAXC) * a.stride;
        if (st) {
          res_d1<V>(a, j, scale_sh, t, vs, ws);
          res_d2<V>(a, j, tix, t, nd, Qs, Ds, trs, vs, ws, a.partials);
        }
        if (!grid_sync(gb, G)) return;
        if (st) {
          final_reduce(a.partials, a.stride, u.tile0, u.ntile, nc, out);
          final_reduce(a.partials + (long long)nc * a.stride, a.stride, u.tile0, u.ntile, nc,
                       out + nc);
          const double inu = 1.0 / beta_sh;
          d2_finish<true>(out, out + nc, nb, nd, j, inu, isn, unit_S(a.S, t.unit),
                          tix == u.tile0, dsc, dsk);
          const double rho = dsc[0];
          for (int k = threadIdx.x; k < nb; k += RSB_BLOCK) {
            const double ck = out[k] / rho, gk = out[nc + k] / rho;
            cv2[k] = k == 0 ? V(ck * isn) : V(ck);
            cv1[k] = k == 0 ? V(gk * isn) : V(gk);
          }
          if (lead) u.alpha[j] = dsc[2];
          __syncthreads();
          res_d3<V>(a, j, tix, t, nd, masked, key, Qs, Ds, trs, vs, ws, cv2, cv1, V(inu / rho),
                    V(1.0 / rho), V(dsc[1] / rho), sm, Pn);
        }
        if (!grid_sync(gb, G)) return;
        if (st) {
          final_reduce(Pn, a.stride, u.tile0, u.ntile, 1, out);
          if (threadIdx.x == 0) {
            const double b = sqrt(out[0]);
            beta_sh = b;
            scale_sh = V(1.0 / b);
            if (lead) u.beta[j + 1] = b;
            if (b <= breakdown * u.dmax && lead) {  // invariant subspace: the cycle ends here
              u.msteps = j + 1;
              u.broke = 1;
            }
          }
          __syncthreads();
          if (beta_sh <= breakdown * u.dmax) msteps = j + 1;
        }
        continue;
      }
      const int nc = 2 + nd + j;
      if (st) res_a<V>(a, j, scale_sh, tix, t, u, Qs, Ds, trs, ws, Pb[ph & 1]);
      if (!grid_sync(gb, G)) return;
      if (st) {
        final_reduce(Pb[ph & 1], a.stride, u.tile0, u.ntile, nc, out);
        res_coef<V>(out, nc, isn, c1, cv1);
        res_b<V>(a, j, tix, t, nd, masked, key, Qs, Ds, trs, ws, cv1, Pb[(ph + 1) & 1]);
      }
      if (!grid_sync(gb, G)) return;
      if (st) {
        final_reduce(Pb[(ph + 1) & 1], a.stride, u.tile0, u.ntile, nc, out);
        res_coef<V>(out, nc, isn, c2, cv2);
        if (tix == u.tile0) {  // column j of S = Q^T L Q
          double* Sm = unit_S(a.S, t.unit);
          for (int k = threadIdx.x; k <= j; k += RSB_BLOCK) {
            const double v = c1[1 + nd + k] + c2[1 + nd + k];
            Sm[k * RSB_MAXM + j] = v;
            Sm[j * RSB_MAXM + k] = v;
          }
        }
        res_c<V>(a, j, tix, t, nd, masked, key, Qs, Ds, trs, ws, cv2, sm, Pb[ph & 1]);
      }
      if (!grid_sync(gb, G)) return;
      if (st) {
        final_reduce(Pb[ph & 1], a.stride, u.tile0, u.ntile, 1, out);
        if (threadIdx.x == 0) {
          const double b = sqrt(out[0]);
          beta_sh = b;
          scale_sh = V(1.0 / b);
          if (lead) u.beta[j + 1] = b;
          if (b <= breakdown * u.dmax && lead) {  // invariant subspace: the cycle ends here
            u.msteps = j + 1;
            u.broke = 1;
          }
        }
        __syncthreads();
        if (beta_sh <= breakdown * u.dmax) msteps = j + 1;
      }
      ++ph;
    }
    for (int uu = blockIdx.x; uu < nunits; uu += G) lz_eig_u<V, true>(a.units[uu], unit_S(a.S, uu), J);
    if (!grid_sync(gb, G)) return;
    res_ritz<V>(a, t, u, Qs, trs, &J.Z[0][0]);
    if (!grid_sync(gb, G)) return;
    lz_resid_t<V, true>(ac, a.Y, 0, tix, sm, out);
    if (!grid_sync(gb, G)) return;
    proj2_t<V, true>(a, a.Y, tix, sm, out);
    if (!grid_sync(gb, G)) return;
    proj3_t<V, true>(a, a.Y, tix, sm, out);
    if (!grid_sync(gb, G)) return;
    if (__ldcg(a.n_active) == 0) break;
  }
}

// Start vector into Y: hash of gid on unit rows (or a given vector), 0 elsewhere.
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_start(LzArgs<V> a, uint64_t sd, const double* from64,
                                                     const float* from32) {
  const Tile t = a.tiles[blockIdx.x];
  const Unit& u = a.units[t.unit];
  if (u.status != U_ACTIVE) return;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    V v = V(0);
    if (unit_has(u, a.ckey, r)) {
      if (from64) v = V(from64[r]);
      else if (from32) v = V(from32[r]);
      else v = V(start_value(sd, a.gid[r]));
    }
    a.Y[r] = v;
  }
}

// ----------------------------------------------------------------------------
// solve set-up per unit
// ----------------------------------------------------------------------------
// mode: number of deflation vectors nd (0, 1, 2).  A unit joins the solve when
// it is valid, its space orthogonal to 1 and the deflation vectors is not
// empty, and (nd > 0) it found a cluster of size nd so far.
// Units whose dimension dim = n - 1 - nd lies outside [dim_lo, dim_hi] are left
// as they are (another solver takes them).
__global__ void k_solve_init(Unit* units, int nunits, int nd, int krylov, int maxcycles, double tol,
                             int require_cluster, int keep, long long dim_lo, long long dim_hi,
                             int* n_active) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nunits) return;
  Unit& u = units[i];
  const long long dim = u.n - 1 - nd;
  if (u.valid && dim > 0 && (dim < dim_lo || dim > dim_hi)) return;
  u.status = U_IDLE;
  if (!u.valid) return;
  if (dim <= 0) return;
  if (require_cluster && u.ncand != nd) return;
  u.nd = nd;
  u.m = (int)min((long long)krylov, dim);
  u.msteps = u.m;
  u.j0 = 0;
  u.kk = 0;
  u.broke = 0;
  u.keep = keep;
  u.cycles = 0;
  u.maxcycles = maxcycles;
  u.tolabs = tol * u.dmax;
  u.inner = 0;
  u.inner_total = 0;
  u.cg_done = 0;
  u.status = U_ACTIVE;
  atomicAdd(n_active, 1);
}

// ----------------------------------------------------------------------------
// host drivers
// ----------------------------------------------------------------------------
template <typename V>
static LzArgs<V> make_args(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units,
                           const uint64_t* ckey, SolveBufs& B) {
  LzArgs<V> a;
  a.slice_ptr = G.slice_ptr;
  a.ent = G.ent;
  a.gid = G.gid;
  a.tiles = tiles;
  a.units = units;
  a.ckey = ckey;
  a.Q = (V*)B.Q;
  a.N = B.N;
  a.W0 = (V*)B.W0;
  a.W1 = (V*)B.W1;
  a.Y = (V*)B.Y;
  a.X = (V*)B.X;
  a.R = (V*)B.R;
  a.P = (V*)B.P;
  a.AP = (V*)B.AP;
  a.D0 = B.D[0];
  a.D1 = B.D[1];
  a.partials = B.partials;
  a.stride = ntiles;
  a.n_active = B.n_active;
  a.stat_cycles = B.stat_cycles;
  a.pb_a = prof_bytes(PROF_LZ_A);
  a.pb_a2 = prof_bytes(PROF_LZ_A2);
  a.pb_b = prof_bytes(PROF_LZ_B);
  a.pb_c = prof_bytes(PROF_LZ_C);
  a.pb_cg = prof_bytes(PROF_CG_AP);
  a.S = B.S;
  a.jmin = B.jmin;
  return a;
}

int solver_setup(Unit* units, int nunits, int nd, int krylov, int maxcycles, double tol,
                 int require_cluster, int keep, SolveBufs& B, cudaStream_t s, long long dim_lo,
                 long long dim_hi) {
  B.maxcycles = maxcycles;
  RSB_CK(cudaMemsetAsync(B.n_active, 0, sizeof(int), s));
  k_solve_init<<<(nunits + 127) / 128, 128, 0, s>>>(units, nunits, nd, krylov, maxcycles, tol,
                                                    require_cluster, keep, dim_lo, dim_hi,
                                                    B.n_active);
  RSB_CKL("k_solve_init");
  return RSB_OK;
}

static int read_active(SolveBufs& B, cudaStream_t s, int* out) {
  RSB_CK(cudaMemcpyAsync(B.h_active, B.n_active, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (B.jmin) RSB_CK(cudaMemcpyAsync(B.h_active + 2, B.jmin, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (B.gb) RSB_CK(cudaMemcpyAsync(B.h_active + 1, &B.gb->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  RSB_CK(cudaStreamSynchronize(s));
  prof_collect();
  *out = *B.h_active;
  if (B.gb && B.h_active[1] == 2)
    return rsb_set_error(RSB_ETIMEOUT,
                         "a bounded device wait gave up and a CTA's bulk copies in flight did "
                         "not drain before it exited");
  if (B.gb && B.h_active[1]) return rsb_set_error(RSB_ETIMEOUT, "a bounded device wait gave up");
  return RSB_OK;
}

template <typename V>
static int lz_start(LzArgs<V>& a, int ntiles, uint64_t sd, const double* from64,
                    const float* from32, cudaStream_t s) {
  k_start<V><<<ntiles, RSB_BLOCK, 0, s>>>(a, sd, from64, from32);
  RSB_CKL("k_start");
  k_lz_resid<V><<<ntiles, RSB_BLOCK, 0, s>>>(a, a.Y, 1);
  RSB_CKL("k_lz_resid(start)");
  k_proj2<V><<<ntiles, RSB_BLOCK, 0, s>>>(a, a.Y);
  RSB_CKL("k_proj2");
  k_proj3<V><<<ntiles, RSB_BLOCK, 0, s>>>(a, a.Y);
  RSB_CKL("k_proj3");
  return RSB_OK;
}

template <typename V>
static int lz_cycle(LzArgs<V>& a, int ntiles, int nunits, int M, double breakdown, GridBar* gb,
                    int trmax, cudaStream_t s) {
  // CTAs per tile of step A1
  const int nsub = std::max(1, (trmax + A1_RPT * RSB_BLOCK - 1) / (A1_RPT * RSB_BLOCK));
  for (int j = 0; j < M; ++j) {
    int pi = prof_before(PROF_LZ_A, s);
    if constexpr (sizeof(V) == 4) {  // FP32: bandwidth-bound; CGS2 with the second pass delayed
      k_lz_a1<V><<<ntiles * nsub, RSB_BLOCK, 0, s>>>(a, j, nsub);
      RSB_CKL("k_lz_a1");
      prof_after(pi, s);
      pi = prof_before(PROF_LZ_A2, s);
      k_lz_d2<V><<<ntiles, RSB_BLOCK, staged_smem<V>(j + 2), s>>>(a, j, gb);
      RSB_CKL("k_lz_d2");
      prof_after(pi, s);
      pi = prof_before(PROF_LZ_B, s);
      k_lz_d3<V><<<ntiles, RSB_BLOCK, 0, s>>>(a, j, breakdown);
      RSB_CKL("k_lz_d3");
      prof_after(pi, s);
      continue;
    }
    // FP64: bound by GB300's FP64 rate; register-streaming kernels, CGS2
    k_lz_a<V><<<ntiles, RSB_BLOCK, 0, s>>>(a, j);
    RSB_CKL("k_lz_a");
    prof_after(pi, s);
    pi = prof_before(PROF_LZ_B, s);
    k_lz_b<V><<<ntiles, RSB_BLOCK, 0, s>>>(a, j);
    RSB_CKL("k_lz_b");
    prof_after(pi, s);
    pi = prof_before(PROF_LZ_C, s);
    k_lz_c<V><<<ntiles, RSB_BLOCK, 0, s>>>(a, j, breakdown);
    RSB_CKL("k_lz_c");
    prof_after(pi, s);
  }
  k_lz_eig<V><<<nunits, RSB_BLOCK, 0, s>>>(a.units, a.S, nunits);
  RSB_CKL("k_lz_eig");
  k_lz_ritz<V><<<ntiles, RSB_BLOCK, 0, s>>>(a);
  RSB_CKL("k_lz_ritz");
  k_lz_resid<V><<<ntiles, RSB_BLOCK, 0, s>>>(a, a.Y, 0);
  RSB_CKL("k_lz_resid");
  k_proj2<V><<<ntiles, RSB_BLOCK, 0, s>>>(a, a.Y);
  RSB_CKL("k_proj2");
  k_proj3<V><<<ntiles, RSB_BLOCK, 0, s>>>(a, a.Y);
  RSB_CKL("k_proj3");
  return RSB_OK;
}

// Runs Lanczos cycles until every participating unit converged or hit its cap.
// The start is the gid hash with seed sd, or from64 / from32 when given.
template <typename V>
static int lanczos_run(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units, int nunits,
                       const uint64_t* ckey, SolveBufs& B, int M, uint64_t sd,
                       const double* from64, const float* from32, int use_graph,
                       cudaStream_t s) {
  LzArgs<V> a = make_args<V>(G, tiles, ntiles, units, ckey, B);
  // step A1 and the resident kernel size their launches by the largest tile
  if (B.trmax <= 0) return rsb_set_error(RSB_EINVAL, "Lanczos solve without its largest tile size");
  int active = 0;
  int rc = read_active(B, s, &active);
  if (rc || active == 0) return rc;
  rc = lz_start<V>(a, ntiles, sd, from64, from32, s);
  if (rc) return rc;
  const double breakdown = 1e-14;
  if (B.gb) {
    // a fresh barrier (count, generation, error word) for this solve; the
    // failure-path test hook starts the count where no CTA sees the last arrival
    RSB_CK(cudaMemsetAsync(B.gb, 0, sizeof(GridBar), s));
    if (g_rsb_poison_barrier && (use_graph == 2 || use_graph == 3))
      RSB_CK(cudaMemsetAsync(&B.gb->count, 0x40, sizeof(unsigned int), s));
  }
  if (use_graph == 3 && B.gb) {
    // the whole solve in one cooperative launch when every tile gets a
    // co-resident CTA holding its rows of the basis; otherwise CUDA graphs
    int dev = 0, nsm = 0, optin = 0, occ = 0;
    RSB_CK(cudaGetDevice(&dev));
    RSB_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    RSB_CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    int trs = B.trmax;
    const size_t smem = res_smem_bytes<V>(M, trs);
    if (smem + 1024 <= (size_t)optin) {  // room for the kernel's static shared memory
      RSB_CK(cudaFuncSetAttribute(k_lz_res<V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
      RSB_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_lz_res<V>, RSB_BLOCK, smem));
      if ((long long)occ * nsm >= ntiles) {
        int maxcyc = B.maxcycles + 1;
        double bd = breakdown;
        GridBar* gb = B.gb;
        LzArgs<V> ar = a;  // the persistent kernel's phases count into one family
        ar.pb_a = ar.pb_a2 = ar.pb_b = ar.pb_c = prof_bytes(PROF_CYCLE);
        void* args[] = {(void*)&ar, (void*)&M, (void*)&trs, (void*)&bd, (void*)&nunits,
                        (void*)&maxcyc, (void*)&gb};
        const int pi = prof_before(PROF_CYCLE, s);
        cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_lz_res<V>, ntiles, RSB_BLOCK,
                                                    args, smem, s);
        rsb_count_launch(1);
        if (e != cudaSuccess) return rsb_set_cuda_error(e, "cudaLaunchCooperativeKernel(k_lz_res)");
        prof_after(pi, s);
        return read_active(B, s, &active);
      }
    }
  }
  if (use_graph == 2 && B.gb) {
    // one persistent cooperative launch per cycle
    int dev = 0, nsm = 0, occ = 0;
    RSB_CK(cudaGetDevice(&dev));
    RSB_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    RSB_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_lz_cycle<V>, RSB_BLOCK, 0));
    const int grid = std::max(1, std::min(ntiles, occ * nsm));
    GridBar* gb = B.gb;
    int jstart = 0;
    LzArgs<V> ar = a;  // the persistent kernel's phases count into one family
    ar.pb_a = ar.pb_a2 = ar.pb_b = ar.pb_c = prof_bytes(PROF_CYCLE);
    for (int cyc = 0; cyc < 100000; ++cyc) {
      RSB_CK(cudaMemsetAsync(B.jmin, 0x7F, sizeof(int), s));
      void* args[] = {(void*)&ar, (void*)&jstart, (void*)&M, (void*)&breakdown, (void*)&ntiles,
                      (void*)&nunits, (void*)&gb};
      const int pi = prof_before(PROF_CYCLE, s);
      cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_lz_cycle<V>, grid, RSB_BLOCK,
                                                  args, 0, s);
      rsb_count_launch(1);
      if (e != cudaSuccess) return rsb_set_cuda_error(e, "cudaLaunchCooperativeKernel(k_lz_cycle)");
      prof_after(pi, s);
      rc = read_active(B, s, &active);
      if (rc || active == 0) break;
      jstart = std::min(std::max(B.h_active[2], 0), M);
    }
    return rc;
  }
  // the staged step D2 (FP32) needs up to 2 * (M + 1) * (RSB_BLOCK + 4) floats of
  // dynamic shared memory (85 KB at M = 40)
  if constexpr (sizeof(V) == 4) {
    RSB_CK(cudaFuncSetAttribute(k_lz_d2<V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)staged_smem<V>(M + 1)));
    // the whole carveout as shared memory: D2 is bound by the CTAs per SM that
    // its staged chunks leave room for (two at the default carveout)
    RSB_CK(cudaFuncSetAttribute(k_lz_d2<V>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                cudaSharedmemCarveoutMaxShared));
  }
  cudaGraphExec_t exec = nullptr;
  std::vector<int> cap_pairs;
  if (use_graph) {
    cudaGraph_t graph = nullptr;
    RSB_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    prof_capture_begin();
    rc = lz_cycle<V>(a, ntiles, nunits, M, breakdown, B.gb, B.trmax, s);
    cap_pairs = prof_capture_end();
    cudaGraph_t g2 = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g2);
    graph = g2;
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return rsb_set_cuda_error(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return rsb_set_cuda_error(e, "cudaGraphInstantiate");
  }
  const char* tr = getenv("RSB_TRACE");
  const bool trace = tr && *tr && *tr != '0';
  auto t_prev = std::chrono::steady_clock::now();
  for (int cyc = 0; cyc < 100000; ++cyc) {
    if (exec) {
      cudaError_t e = cudaGraphLaunch(exec, s);
      rsb_count_launch(3 * M + 5);  // the kernels of one cycle
      if (e != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        return rsb_set_cuda_error(e, "cudaGraphLaunch");
      }
      prof_replay(cap_pairs);
    } else {
      rc = lz_cycle<V>(a, ntiles, nunits, M, breakdown, B.gb, B.trmax, s);
      if (rc) return rc;
    }
    rc = read_active(B, s, &active);
    if (trace) {  // per-cycle wall time and units still active (RSB_TRACE=1)
      const auto now = std::chrono::steady_clock::now();
      fprintf(stderr, "[rsb]   %9.3f ms    cycle %d: %d of %d units active\n",
              std::chrono::duration<double, std::milli>(now - t_prev).count(), cyc, active,
              nunits);
      t_prev = now;
    }
    if (rc || active == 0) break;
  }
  if (exec) cudaGraphExecDestroy(exec);
  return rc;
}

int solver_lanczos(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units, int nunits,
                   const uint64_t* ckey, SolveBufs& B, int f32, int M, uint64_t sd,
                   const double* from64, const float* from32, int use_graph, cudaStream_t s) {
  if (ntiles <= 0 || nunits <= 0) return RSB_OK;
  if (f32)
    return lanczos_run<float>(G, tiles, ntiles, units, nunits, ckey, B, M, sd, from64, from32,
                              use_graph, s);
  return lanczos_run<double>(G, tiles, ntiles, units, nunits, ckey, B, M, sd, from64, from32,
                             use_graph, s);
}

// ----------------------------------------------------------------------------
// inverse iteration with CG
// ----------------------------------------------------------------------------
// CG init from w0 / beta0: x = 0, r = p = b, rr = ||b||^2.
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_cg_init(LzArgs<V> a) {
  __shared__ double sm[RSB_WARPS];
  __shared__ double out[1];
  const Tile t = a.tiles[blockIdx.x];
  Unit& u = a.units[t.unit];
  if (u.status != U_ACTIVE) return;
  const V s = V(1.0 / u.beta0);
  Acc<V> acc;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    const V b = s * a.W0[r];
    a.X[r] = V(0);
    a.R[r] = b;
    a.P[r] = b;
    acc.add(b * b);
  }
  const double sum = block_sum(acc.get(), sm);
  if (threadIdx.x == 0) a.partials[blockIdx.x] = sum;
  if (last_cta(&u.cnt, u.ntile)) {
    final_reduce(a.partials, a.stride, u.tile0, u.ntile, 1, out);
    if (threadIdx.x == 0) {
      u.rr = out[0];
      u.bnorm = sqrt(out[0]);
      u.inner = 0;
      u.cg_done = 0;
    }
  }
}

// AP = L P, pAp -> alpha
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_cg_ap(LzArgs<V> a) {
  __shared__ double sm[RSB_WARPS];
  __shared__ double out[1];
  const Tile t = a.tiles[blockIdx.x];
  Unit& u = a.units[t.unit];
  if (u.status != U_ACTIVE || u.cg_done) return;
  Acc<V> acc;
  unsigned long long pbytes = 0;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    const V pr = a.P[r];
    const V ap = spmv_row_ro<V>(a.slice_ptr, a.ent, a.P, r, pr);
    a.AP[r] = ap;
    acc.add(pr * ap);
    if (a.pb_cg) pbytes += 4ull * row_width(a.slice_ptr, r) + 2ull * sizeof(V);
  }
  if (a.pb_cg) prof_add(a.pb_cg, pbytes);
  const double sum = block_sum(acc.get(), sm);
  if (threadIdx.x == 0) a.partials[blockIdx.x] = sum;
  if (last_cta(&u.cnt, u.ntile)) {
    final_reduce(a.partials, a.stride, u.tile0, u.ntile, 1, out);
    if (threadIdx.x == 0) u.cg_alpha = u.rr / out[0];
  }
}

// x += alpha p, r -= alpha Ap; sums for ||r||^2 and the projection of r.
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_cg_xr(LzArgs<V> a, double cg_tol, int cg_maxit,
                                                     int* n_cg) {
  __shared__ double sm[RSB_WARPS];
  __shared__ double out[2 + RSB_MAXD];
  const Tile t = a.tiles[blockIdx.x];
  Unit& u = a.units[t.unit];
  if (u.status != U_ACTIVE || u.cg_done) return;
  const int nd = u.nd;
  const V al = V(u.cg_alpha);
  Acc<V> r2, rs, d0, d1;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    a.X[r] += al * a.P[r];
    const V rr = a.R[r] - al * a.AP[r];
    a.R[r] = rr;
    r2.add(rr * rr);
    rs.add(rr);
    if (nd > 0) d0.add(V(a.D0[r]) * rr);
    if (nd > 1) d1.add(V(a.D1[r]) * rr);
  }
  double v[4] = {r2.get(), rs.get(), d0.get(), d1.get()};
  const int nv = 2 + nd;
  for (int c = 0; c < nv; ++c) {
    const double sum = block_sum(v[c], sm);
    if (threadIdx.x == 0) a.partials[(long long)c * a.stride + blockIdx.x] = sum;
  }
  if (last_cta(&u.cnt, u.ntile)) {
    final_reduce(a.partials, a.stride, u.tile0, u.ntile, nv, out);
    if (threadIdx.x == 0) {
      double cp2 = 0.0;
      u.cp[0] = out[1] * u.isn;
      cp2 += u.cp[0] * u.cp[0];
      for (int l = 0; l < nd; ++l) {
        u.cp[1 + l] = out[2 + l];
        cp2 += u.cp[1 + l] * u.cp[1 + l];
      }
      const double rrn = fmax(out[0] - cp2, 0.0);
      u.inner += 1;
      u.inner_total += 1;
      if (sqrt(rrn) <= cg_tol * u.bnorm || u.inner >= cg_maxit) {
        u.cg_done = 1;
        atomicSub(n_cg, 1);
      } else {
        u.cg_beta = rrn / u.rr;
        u.rr = rrn;
      }
    }
  }
}

// r -= B cp (projection), p = r + beta p while CG continues.
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_cg_p(LzArgs<V> a) {
  const Tile t = a.tiles[blockIdx.x];
  const Unit& u = a.units[t.unit];
  if (u.status != U_ACTIVE || u.cg_done) return;
  const int nd = u.nd;
  const V be = V(u.cg_beta);
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    V v = a.R[r];
    if (unit_has(u, a.ckey, r)) v -= V(u.cp[0] * u.isn);
    if (nd > 0) v -= V(u.cp[1]) * V(a.D0[r]);
    if (nd > 1) v -= V(u.cp[2]) * V(a.D1[r]);
    a.R[r] = v;
    a.P[r] = v + be * a.P[r];
  }
}

// ----------------------------------------------------------------------------
// Flexible CG (§7): the first direction is the residual itself, later ones the
// AMG-preconditioned residual z; beta = z.(r - r_old) / (z_old . r_old).  With
// u.rr holding z.r, k_cg_ap gives alpha = z.r / p.Ap as in plain CG.
// ----------------------------------------------------------------------------
// x += alpha p; r_old = r (in W1); r -= alpha Ap; sums for ||r||^2 and the
// projection of r; convergence as in plain CG.
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_fcg_xr(LzArgs<V> a, double cg_tol, int cg_maxit,
                                                      int* n_cg) {
  __shared__ double sm[RSB_WARPS];
  __shared__ double out[2 + RSB_MAXD];
  const Tile t = a.tiles[blockIdx.x];
  Unit& u = a.units[t.unit];
  if (u.status != U_ACTIVE || u.cg_done) return;
  const int nd = u.nd;
  const V al = V(u.cg_alpha);
  Acc<V> r2, rs, d0, d1;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    a.X[r] += al * a.P[r];
    const V ro = a.R[r];
    const V rr = ro - al * a.AP[r];
    a.W1[r] = ro;
    a.R[r] = rr;
    r2.add(rr * rr);
    rs.add(rr);
    if (nd > 0) d0.add(V(a.D0[r]) * rr);
    if (nd > 1) d1.add(V(a.D1[r]) * rr);
  }
  double v[4] = {r2.get(), rs.get(), d0.get(), d1.get()};
  const int nv = 2 + nd;
  for (int c = 0; c < nv; ++c) {
    const double sum = block_sum(v[c], sm);
    if (threadIdx.x == 0) a.partials[(long long)c * a.stride + blockIdx.x] = sum;
  }
  if (last_cta(&u.cnt, u.ntile)) {
    final_reduce(a.partials, a.stride, u.tile0, u.ntile, nv, out);
    if (threadIdx.x == 0) {
      double cp2 = 0.0;
      u.cp[0] = out[1] * u.isn;
      cp2 += u.cp[0] * u.cp[0];
      for (int l = 0; l < nd; ++l) {
        u.cp[1 + l] = out[2 + l];
        cp2 += u.cp[1 + l] * u.cp[1 + l];
      }
      const double rrn = fmax(out[0] - cp2, 0.0);
      u.inner += 1;
      u.inner_total += 1;
      if (sqrt(rrn) <= cg_tol * u.bnorm || u.inner >= cg_maxit) {
        u.cg_done = 1;
        atomicSub(n_cg, 1);
      }
    }
  }
}

// r -= B cp (projection): the residual the preconditioner sees
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_fcg_proj(LzArgs<V> a) {
  const Tile t = a.tiles[blockIdx.x];
  const Unit& u = a.units[t.unit];
  if (u.status != U_ACTIVE || u.cg_done) return;
  const int nd = u.nd;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    V v = a.R[r];
    if (unit_has(u, a.ckey, r)) v -= V(u.cp[0] * u.isn);
    if (nd > 0) v -= V(u.cp[1]) * V(a.D0[r]);
    if (nd > 1) v -= V(u.cp[2]) * V(a.D1[r]);
    a.R[r] = v;
  }
}

// z (in Y) restricted to the unit's rows; z.r, z.r_old and the projection sums of z
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_fcg_z(LzArgs<V> a) {
  __shared__ double sm[RSB_WARPS];
  __shared__ double out[3 + RSB_MAXD];
  const Tile t = a.tiles[blockIdx.x];
  Unit& u = a.units[t.unit];
  if (u.status != U_ACTIVE || u.cg_done) return;
  const int nd = u.nd;
  Acc<V> zr, zo, zs, d0, d1;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    V z = a.Y[r];
    if (!unit_has(u, a.ckey, r)) {
      z = V(0);
      a.Y[r] = z;
    }
    zr.add(z * a.R[r]);
    zo.add(z * a.W1[r]);
    zs.add(z);
    if (nd > 0) d0.add(V(a.D0[r]) * z);
    if (nd > 1) d1.add(V(a.D1[r]) * z);
  }
  double v[5] = {zr.get(), zo.get(), zs.get(), d0.get(), d1.get()};
  const int nv = 3 + nd;
  for (int c = 0; c < nv; ++c) {
    const double sum = block_sum(v[c], sm);
    if (threadIdx.x == 0) a.partials[(long long)c * a.stride + blockIdx.x] = sum;
  }
  if (last_cta(&u.cnt, u.ntile)) {
    final_reduce(a.partials, a.stride, u.tile0, u.ntile, nv, out);
    if (threadIdx.x == 0) {
      u.fz_rz = out[0];
      u.fz_ro = out[1];
      u.cz[0] = out[2] * u.isn;
      for (int l = 0; l < nd; ++l) u.cz[1 + l] = out[3 + l];
    }
  }
}

// z -= B cz; p = z + beta p with the flexible beta; z.r becomes the new rr
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_fcg_p(LzArgs<V> a) {
  const Tile t = a.tiles[blockIdx.x];
  Unit& u = a.units[t.unit];
  if (u.status != U_ACTIVE || u.cg_done) return;
  const int nd = u.nd;
  const double rz = u.fz_rz;
  const V be = V((rz - u.fz_ro) / u.rr);
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    V z = a.Y[r];
    if (unit_has(u, a.ckey, r)) z -= V(u.cz[0] * u.isn);
    if (nd > 0) z -= V(u.cz[1]) * V(a.D0[r]);
    if (nd > 1) z -= V(u.cz[2]) * V(a.D1[r]);
    a.P[r] = z + be * a.P[r];
  }
  // every CTA of the unit has read u.rr above; the unit's rr is rewritten by
  // the next launch that needs it (k_fcg_rr), after this kernel has finished
}

template <typename V>
__global__ void k_fcg_rr(Unit* units, int nunits) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nunits) return;
  Unit& u = units[i];
  if (u.status != U_ACTIVE || u.cg_done) return;
  u.rr = u.fz_rz;
}

// Outer step: y = x; Ly, yLy, yy -> Rayleigh quotient.
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_inv_rq(LzArgs<V> a) {
  __shared__ double sm[RSB_WARPS];
  __shared__ double out[2];
  const Tile t = a.tiles[blockIdx.x];
  Unit& u = a.units[t.unit];
  if (u.status != U_ACTIVE) return;
  Acc<V> yly, yy;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    const V yr = a.X[r];
    const V ly = spmv_row_ro<V>(a.slice_ptr, a.ent, a.X, r, yr);
    a.AP[r] = ly;
    yly.add(yr * ly);
    yy.add(yr * yr);
  }
  double v[2] = {yly.get(), yy.get()};
  for (int c = 0; c < 2; ++c) {
    const double sum = block_sum(v[c], sm);
    if (threadIdx.x == 0) a.partials[(long long)c * a.stride + blockIdx.x] = sum;
  }
  if (last_cta(&u.cnt, u.ntile)) {
    final_reduce(a.partials, a.stride, u.tile0, u.ntile, 2, out);
    if (threadIdx.x == 0) {
      u.theta = out[0] / out[1];
      u.ynorm2 = out[1];
    }
  }
}

// Outer step: residual ||Ly - lambda y|| / ||y||, stop tests, projection dots
// of y for the next right-hand side.
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_inv_res(LzArgs<V> a, int max_outer, int refine) {
  __shared__ double sm[RSB_WARPS];
  __shared__ double out[2 + RSB_MAXD];
  const Tile t = a.tiles[blockIdx.x];
  Unit& u = a.units[t.unit];
  if (u.status != U_ACTIVE) return;
  const int nd = u.nd;
  const V th = V(u.theta);
  Acc<V> r2, ys, d0, d1;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    const V yr = a.X[r];
    const V res = a.AP[r] - th * yr;
    r2.add(res * res);
    ys.add(yr);
    if (nd > 0) d0.add(V(a.D0[r]) * yr);
    if (nd > 1) d1.add(V(a.D1[r]) * yr);
  }
  double v[4] = {r2.get(), ys.get(), d0.get(), d1.get()};
  const int nv = 2 + nd;
  for (int c = 0; c < nv; ++c) {
    const double sum = block_sum(v[c], sm);
    if (threadIdx.x == 0) a.partials[(long long)c * a.stride + blockIdx.x] = sum;
  }
  if (last_cta(&u.cnt, u.ntile)) {
    final_reduce(a.partials, a.stride, u.tile0, u.ntile, nv, out);
    if (threadIdx.x == 0) {
      u.resid = sqrt(out[0] / u.ynorm2);
      u.cp[0] = out[1] * u.isn;
      for (int l = 0; l < nd; ++l) u.cp[1 + l] = out[2 + l];
      if (refine) {
        u.status = u.resid <= u.tolabs ? U_CONVERGED : U_CAPPED;
        atomicSub(a.n_active, 1);
        return;
      }
      u.cycles += 1;
      atomicAdd((unsigned long long*)a.stat_cycles, 1ull);
      int st = U_ACTIVE;
      if (u.resid <= u.tolabs || u.inner == 1) st = U_CONVERGED;
      else if (u.cycles >= max_outer) st = U_CAPPED;
      if (st != U_ACTIVE) {
        u.status = st;
        atomicSub(a.n_active, 1);
      }
    }
  }
}

__global__ void k_count_cg(Unit* units, int nunits, int* n_cg) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nunits && units[i].status == U_ACTIVE && !units[i].cg_done) atomicAdd(n_cg, 1);
}

int amg_setup(int f32, const LevelGraph& G, const Tile* tiles, int ntiles, const Unit* units,
              const std::vector<Unit>& hunits, cudaStream_t s);
int amg_apply(int f32, const LevelGraph& G, const Tile* tiles, int ntiles, const Unit* units,
              const void* r, void* z, cudaStream_t s);

template <typename V>
static int cg_block(LzArgs<V>& a, int ntiles, int iters, double cg_tol, int cg_maxit, int* n_cg,
                    cudaStream_t s, const LevelGraph* amgG = nullptr, int nunits = 0) {
  for (int i = 0; i < iters; ++i) {
    const int pi = prof_before(PROF_CG_AP, s);
    k_cg_ap<V><<<ntiles, RSB_BLOCK, 0, s>>>(a);
    RSB_CKL("k_cg_ap");
    prof_after(pi, s);
    if (!amgG) {
      k_cg_xr<V><<<ntiles, RSB_BLOCK, 0, s>>>(a, cg_tol, cg_maxit, n_cg);
      RSB_CKL("k_cg_xr");
      k_cg_p<V><<<ntiles, RSB_BLOCK, 0, s>>>(a);
      RSB_CKL("k_cg_p");
      continue;
    }
    // flexible CG preconditioned by one AMG V-cycle (§7)
    k_fcg_xr<V><<<ntiles, RSB_BLOCK, 0, s>>>(a, cg_tol, cg_maxit, n_cg);
    RSB_CKL("k_fcg_xr");
    k_fcg_proj<V><<<ntiles, RSB_BLOCK, 0, s>>>(a);
    RSB_CKL("k_fcg_proj");
    const int pv = prof_before(PROF_AMG, s);
    int rc = amg_apply(sizeof(V) == 4, *amgG, a.tiles, ntiles, a.units, a.R, a.Y, s);
    if (rc) return rc;
    prof_after(pv, s);
    k_fcg_z<V><<<ntiles, RSB_BLOCK, 0, s>>>(a);
    RSB_CKL("k_fcg_z");
    k_fcg_p<V><<<ntiles, RSB_BLOCK, 0, s>>>(a);
    RSB_CKL("k_fcg_p");
    k_fcg_rr<V><<<(nunits + 127) / 128, 128, 0, s>>>(a.units, nunits);
    RSB_CKL("k_fcg_rr");
  }
  return RSB_OK;
}

template <typename V>
static int inverse_run(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units, int nunits,
                       const uint64_t* ckey, SolveBufs& B, uint64_t sd, const double* from64,
                       const float* from32, double cg_tol, int cg_maxit, int max_outer,
                       int use_graph, int64_t* inner_out, cudaStream_t s,
                       const std::vector<Unit>* amg_units) {
  LzArgs<V> a = make_args<V>(G, tiles, ntiles, units, ckey, B);
  // step A1 and the resident kernel size their launches by the largest tile
  if (B.trmax <= 0) return rsb_set_error(RSB_EINVAL, "Lanczos solve without its largest tile size");
  int active = 0;
  int rc = read_active(B, s, &active);
  if (rc || active == 0) return rc;
  rc = lz_start<V>(a, ntiles, sd, from64, from32, s);  // W0 = projected start, beta0
  if (rc) return rc;
  const LevelGraph* amgG = nullptr;
  if (amg_units) {  // the hierarchy of every unit of the level (§7)
    if ((rc = amg_setup(sizeof(V) == 4, G, tiles, ntiles, units, *amg_units, s))) return rc;
    amgG = &G;
  }
  const int CGK = 8;
  cudaGraphExec_t exec = nullptr;
  std::vector<int> cap_pairs;
  if (use_graph) {
    cudaGraph_t graph = nullptr;
    RSB_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    prof_capture_begin();
    rc = cg_block<V>(a, ntiles, CGK, cg_tol, cg_maxit, B.n_cg, s, amgG, nunits);
    cap_pairs = prof_capture_end();
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return rsb_set_cuda_error(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return rsb_set_cuda_error(e, "cudaGraphInstantiate");
  }
  for (int outer = 0; outer < max_outer + 1 && active > 0; ++outer) {
    k_cg_init<V><<<ntiles, RSB_BLOCK, 0, s>>>(a);
    RSB_CKL("k_cg_init");
    RSB_CK(cudaMemsetAsync(B.n_cg, 0, sizeof(int), s));
    k_count_cg<<<(nunits + 127) / 128, 128, 0, s>>>(units, nunits, B.n_cg);
    RSB_CKL("k_count_cg");
    for (int blk = 0; blk < cg_maxit / CGK + 2; ++blk) {
      if (exec) {
        cudaError_t e = cudaGraphLaunch(exec, s);
        rsb_count_launch((amgG ? 7 + 13 * 20 : 3) * CGK);
        if (e != cudaSuccess) {
          cudaGraphExecDestroy(exec);
          return rsb_set_cuda_error(e, "cudaGraphLaunch");
        }
        prof_replay(cap_pairs);
      } else {
        rc = cg_block<V>(a, ntiles, CGK, cg_tol, cg_maxit, B.n_cg, s, amgG, nunits);
        if (rc) break;
      }
      int ncg = 0;
      RSB_CK(cudaMemcpyAsync(B.h_active, B.n_cg, sizeof(int), cudaMemcpyDeviceToHost, s));
      RSB_CK(cudaStreamSynchronize(s));
      prof_collect();
      ncg = *B.h_active;
      if (ncg <= 0) break;
    }
    if (rc) break;
    k_inv_rq<V><<<ntiles, RSB_BLOCK, 0, s>>>(a);
    RSB_CKL("k_inv_rq");
    k_inv_res<V><<<ntiles, RSB_BLOCK, 0, s>>>(a, max_outer, 0);
    RSB_CKL("k_inv_res");
    rc = read_active(B, s, &active);
    if (rc || active == 0) break;
    // next right-hand side: x projected (second pass) and normalised into W0
    k_proj2<V><<<ntiles, RSB_BLOCK, 0, s>>>(a, a.X);
    RSB_CKL("k_proj2");
    k_proj3<V><<<ntiles, RSB_BLOCK, 0, s>>>(a, a.X);
    RSB_CKL("k_proj3");
  }
  if (exec) cudaGraphExecDestroy(exec);
  (void)inner_out;
  return rc;
}

int solver_inverse(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units, int nunits,
                   const uint64_t* ckey, SolveBufs& B, int f32, uint64_t sd, const double* from64,
                   const float* from32, double cg_tol, int cg_maxit, int max_outer, int use_graph,
                   cudaStream_t s, const std::vector<Unit>* amg_units) {
  if (ntiles <= 0 || nunits <= 0) return RSB_OK;
  if (f32)
    return inverse_run<float>(G, tiles, ntiles, units, nunits, ckey, B, sd, from64, from32, cg_tol,
                              cg_maxit, max_outer, use_graph, nullptr, s, amg_units);
  return inverse_run<double>(G, tiles, ntiles, units, nunits, ckey, B, sd, from64, from32, cg_tol,
                             cg_maxit, max_outer, use_graph, nullptr, s, amg_units);
}

// ----------------------------------------------------------------------------
// FP64 Rayleigh-quotient refinement of an FP32 vector (mixed precision):
// y = FP64 copy of the FP32 vector, theta = y^T L y / y^T y and the residual
// ||L y - theta y|| / ||y|| in FP64; the FP64 y lands in B.X.
// ----------------------------------------------------------------------------
int solver_rq_refine(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units, int nunits,
                     const uint64_t* ckey, SolveBufs& B, const float* from32, cudaStream_t s) {
  if (ntiles <= 0 || nunits <= 0) return RSB_OK;
  SolveBufs Bx = B;
  Bx.Y = B.X;  // k_start writes a.Y; the refinement kernels read a.X
  LzArgs<double> a = make_args<double>(G, tiles, ntiles, units, ckey, Bx);
  k_start<double><<<ntiles, RSB_BLOCK, 0, s>>>(a, 0ull, nullptr, from32);
  RSB_CKL("k_start(refine)");
  k_inv_rq<double><<<ntiles, RSB_BLOCK, 0, s>>>(a);
  RSB_CKL("k_inv_rq(refine)");
  k_inv_res<double><<<ntiles, RSB_BLOCK, 0, s>>>(a, 0, 1);
  RSB_CKL("k_inv_res(refine)");
  (void)nunits;
  return RSB_OK;
}

// ----------------------------------------------------------------------------
// result vector: out = y / ||y|| (FP64), for units that took part in the solve
// ----------------------------------------------------------------------------
// better_only: a polish result, written only where its residual is below the
// one recorded for candidate cand (the refined stage-1 vector already in out);
// k_keep_better then settles the unit's record.
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_write_vec(LzArgs<V> a, const V* __restrict__ y,
                                                         double* out, int cand, int better_only) {
  const Tile t = a.tiles[blockIdx.x];
  Unit& u = a.units[t.unit];
  if (u.status != U_CONVERGED && u.status != U_CAPPED) return;
  if (better_only && !(u.resid < u.res[cand])) return;
  const double sc = 1.0 / sqrt(u.ynorm2);
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) out[r] = sc * (double)y[r];
  if (!better_only && blockIdx.x == u.tile0 && threadIdx.x == 0 && cand >= 0) {
    u.lam[cand] = u.theta;
    u.res[cand] = u.resid;
  }
}

// After a polish: the unit keeps the smaller-residual of the refined stage-1
// vector and the polished one (a capped polish can end on a Ritz vector whose
// residual exceeds its start's); it counts as converged at tol1 * dmax.
__global__ void k_keep_better(Unit* units, int nunits, int cand, double tol1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nunits) return;
  Unit& u = units[i];
  if (u.status != U_CONVERGED && u.status != U_CAPPED) return;
  if (u.resid < u.res[cand]) {
    u.lam[cand] = u.theta;
    u.res[cand] = u.resid;
  } else {
    u.theta = u.lam[cand];
    u.resid = u.res[cand];
  }
  u.status = u.resid <= tol1 * u.dmax ? U_CONVERGED : U_CAPPED;
}

int solver_write_vector(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units,
                        const uint64_t* ckey, SolveBufs& B, int f32, int from_x, double* out,
                        int cand, int better_only, cudaStream_t s) {
  if (ntiles <= 0) return RSB_OK;
  if (f32) {
    LzArgs<float> a = make_args<float>(G, tiles, ntiles, units, ckey, B);
    k_write_vec<float><<<ntiles, RSB_BLOCK, 0, s>>>(a, from_x ? a.X : a.Y, out, cand, better_only);
  } else {
    LzArgs<double> a = make_args<double>(G, tiles, ntiles, units, ckey, B);
    k_write_vec<double><<<ntiles, RSB_BLOCK, 0, s>>>(a, from_x ? a.X : a.Y, out, cand,
                                                     better_only);
  }
  RSB_CKL("k_write_vec");
  return RSB_OK;
}

int solver_keep_better(Unit* units, int nunits, int cand, double tol1, cudaStream_t s) {
  k_keep_better<<<(nunits + 127) / 128, 128, 0, s>>>(units, nunits, cand, tol1);
  RSB_CKL("k_keep_better");
  return RSB_OK;
}

// ----------------------------------------------------------------------------
// R5: rotation of a 2- or 3-dimensional cluster basis minimising sum (U R)^4
// ----------------------------------------------------------------------------
// Moments M[a][b][c][d] = sum_r U_a U_b U_c U_d over unit rows, stored for
// a <= b <= c <= d (15 for three columns); the rotation is then found from the
// tensor alone by cyclic pairwise steps, each the closed-form optimum of a
// 2-D rotation (maximise sum (x' y')^2).
__device__ __forceinline__ int mom_index(int a, int b, int c, int d) {
  // sort a<=b<=c<=d then enumerate combinations with repetition of {0,1,2}
  int v[4] = {a, b, c, d};
  for (int i = 0; i < 4; ++i)
    for (int j = i + 1; j < 4; ++j)
      if (v[j] < v[i]) { const int t = v[i]; v[i] = v[j]; v[j] = t; }
  int idx = 0;
  for (int p = 0; p < 3; ++p)
    for (int q = p; q < 3; ++q)
      for (int r = q; r < 3; ++r)
        for (int s = r; s < 3; ++s) {
          if (p == v[0] && q == v[1] && r == v[2] && s == v[3]) return idx;
          ++idx;
        }
  return 0;
}

__global__ void __launch_bounds__(RSB_BLOCK)
    k_quartic_moments(const Tile* __restrict__ tiles, Unit* units, const uint64_t* __restrict__ ckey,
                      const double* __restrict__ v0, const double* __restrict__ v1,
                      const double* __restrict__ v2, double* partials, long long stride,
                      double* mom) {
  __shared__ double sm[RSB_WARPS];
  __shared__ double out[15];
  const Tile t = tiles[blockIdx.x];
  Unit& u = units[t.unit];
  if (!u.valid || u.ncand < 2) return;
  const int m = u.ncand;
  double acc[15];
  for (int i = 0; i < 15; ++i) acc[i] = 0.0;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    if (!unit_has(u, ckey, r)) continue;
    const double x[3] = {v0[r], v1[r], m > 2 ? v2[r] : 0.0};
    int idx = 0;
    for (int p = 0; p < 3; ++p)
      for (int q = p; q < 3; ++q)
        for (int rr = q; rr < 3; ++rr)
          for (int s = rr; s < 3; ++s) acc[idx++] += x[p] * x[q] * x[rr] * x[s];
  }
  for (int c = 0; c < 15; ++c) {
    const double sum = block_sum(acc[c], sm);
    if (threadIdx.x == 0) partials[(long long)c * stride + blockIdx.x] = sum;
  }
  if (last_cta(&u.cnt, u.ntile)) {
    final_reduce(partials, stride, u.tile0, u.ntile, 15, out);
    if (threadIdx.x < 15) mom[(long long)t.unit * 24 + threadIdx.x] = out[threadIdx.x];
  }
}

// S(p,q; i) = sum_r x^(4-i) y^i with x = U R[:,p], y = U R[:,q], from the full
// (81-entry) moment tensor Mf.
__device__ double rot_moment(const double* Mf, const double* R, int p, int q, int i) {
  double s = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double fa = R[a * 3 + (0 < 4 - i ? p : q)];
    for (int b = 0; b < 3; ++b) {
      const double fab = fa * R[b * 3 + (1 < 4 - i ? p : q)];
      for (int c = 0; c < 3; ++c) {
        const double fabc = fab * R[c * 3 + (2 < 4 - i ? p : q)];
        const double* row = Mf + ((a * 3 + b) * 3 + c) * 3;
        const int col = 3 < 4 - i ? p : q;
        s += fabc * (row[0] * R[0 * 3 + col] + row[1] * R[1 * 3 + col] + row[2] * R[2 * 3 + col]);
      }
    }
  }
  return s;
}

__global__ void k_quartic_rotation(Unit* units, int nunits, double* mom) {
  const int ui = blockIdx.x * blockDim.x + threadIdx.x;
  if (ui >= nunits) return;
  Unit& u = units[ui];
  if (!u.valid || u.ncand < 2) return;
  const int m = u.ncand;
  double* M = mom + (long long)ui * 24;
  double Mf[81];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) Mf[((a * 3 + b) * 3 + c) * 3 + d] = M[mom_index(a, b, c, d)];
  double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  const int sweeps = m > 2 ? 50 : 1;
  for (int sw = 0; sw < sweeps; ++sw) {
    double dmax = 0.0;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double x4 = rot_moment(Mf, R, p, q, 0);
        const double x3y = rot_moment(Mf, R, p, q, 1);
        const double x2y2 = rot_moment(Mf, R, p, q, 2);
        const double xy3 = rot_moment(Mf, R, p, q, 3);
        const double y4 = rot_moment(Mf, R, p, q, 4);
        // u = x^2 - y^2, w = 2 x y
        const double uu = x4 - 2.0 * x2y2 + y4;
        const double ww = 4.0 * x2y2;
        const double uw = 2.0 * (x3y - xy3);
        const double th = 0.25 * atan2(uw, 0.5 * (ww - uu));
        const double c = cos(th), s = sin(th);
        for (int a = 0; a < 3; ++a) {
          const double rp = R[a * 3 + p], rq = R[a * 3 + q];
          R[a * 3 + p] = c * rp - s * rq;
          R[a * 3 + q] = s * rp + c * rq;
        }
        dmax = fmax(dmax, fabs(th));
      }
    if (dmax < 1e-12) break;
  }
  for (int i = 0; i < 9; ++i) M[15 + i] = R[i];
}

__global__ void __launch_bounds__(RSB_BLOCK)
    k_quartic_apply(const Tile* __restrict__ tiles, const Unit* units, double* v0, double* v1,
                    double* v2, const double* mom) {
  const Tile t = tiles[blockIdx.x];
  const Unit& u = units[t.unit];
  if (!u.valid || u.ncand < 2) return;
  const int m = u.ncand;
  const double* R = mom + (long long)t.unit * 24 + 15;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    const double x[3] = {v0[r], v1[r], m > 2 ? v2[r] : 0.0};
    double y[3];
    for (int c = 0; c < m; ++c) {
      double s = 0.0;
      for (int a = 0; a < m; ++a) s += x[a] * R[a * 3 + c];
      y[c] = s;
    }
    v0[r] = y[0];
    v1[r] = y[1];
    if (m > 2) v2[r] = y[2];
  }
}

int solver_quartic(const Tile* tiles, int ntiles, Unit* units, int nunits, const uint64_t* ckey,
                   double* v0, double* v1, double* v2, double* partials, double* mom,
                   cudaStream_t s) {
  if (ntiles <= 0) return RSB_OK;
  k_quartic_moments<<<ntiles, RSB_BLOCK, 0, s>>>(tiles, units, ckey, v0, v1, v2, partials, ntiles,
                                                 mom);
  RSB_CKL("k_quartic_moments");
  k_quartic_rotation<<<(nunits + 63) / 64, 64, 0, s>>>(units, nunits, mom);
  RSB_CKL("k_quartic_rotation");
  k_quartic_apply<<<ntiles, RSB_BLOCK, 0, s>>>(tiles, units, v0, v1, v2, mom);
  RSB_CKL("k_quartic_apply");
  return RSB_OK;
}

// ----------------------------------------------------------------------------
// cluster test after a deflated solve (R5): candidate nd joins when its
// eigenvalue is within cluster_tol * lambda_a of the first.
// ----------------------------------------------------------------------------
__global__ void k_cluster_check(Unit* units, int nunits, int nd, double cluster_tol) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nunits) return;
  Unit& u = units[i];
  if (!u.valid || u.ncand != nd) return;
  if (u.status != U_CONVERGED && u.status != U_CAPPED) return;
  if (fabs(u.lam[nd] - u.lam[0]) <= cluster_tol * u.lam[0]) u.ncand = nd + 1;
}

int solver_cluster_check(Unit* units, int nunits, int nd, double cluster_tol, cudaStream_t s) {
  k_cluster_check<<<(nunits + 127) / 128, 128, 0, s>>>(units, nunits, nd, cluster_tol);
  RSB_CKL("k_cluster_check");
  return RSB_OK;
}

// Statistics of the finished solve: count capped units, max residual / dmax.
__global__ void k_solve_stats(const Unit* units, int nunits, int* capped, double* resid_max,
                              int cand) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nunits) return;
  const Unit& u = units[i];
  if (u.status == U_CAPPED) atomicAdd(capped, 1);
  if (u.status == U_CONVERGED || u.status == U_CAPPED) {
    const double r = u.resid / fmax(u.dmax, 1e-300);
    // non-negative doubles order like their bit patterns
    atomicMax((unsigned long long*)resid_max, (unsigned long long)__double_as_longlong(r));
  }
  (void)cand;
}

// CG iterations of the inverse-iteration solve just finished, summed over units
__global__ void k_sum_inner(const Unit* units, int nunits, long long* inner) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nunits) return;
  const Unit& u = units[i];
  if (u.status == U_CONVERGED || u.status == U_CAPPED)
    atomicAdd((unsigned long long*)inner, (unsigned long long)u.inner_total);
}

int solver_sum_inner(const Unit* units, int nunits, long long* inner, cudaStream_t s) {
  k_sum_inner<<<(nunits + 127) / 128, 128, 0, s>>>(units, nunits, inner);
  RSB_CKL("k_sum_inner");
  return RSB_OK;
}

int solver_stats(const Unit* units, int nunits, int* capped, double* resid_max, cudaStream_t s) {
  k_solve_stats<<<(nunits + 127) / 128, 128, 0, s>>>(units, nunits, capped, resid_max, 0);
  RSB_CKL("k_solve_stats");
  return RSB_OK;
}
