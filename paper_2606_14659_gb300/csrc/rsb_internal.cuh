// rsb_internal.cuh — shared layout, device helpers and launcher declarations of
// librsb.  Everything here is private to the library; the public surface is
// include/rsb.h.
//
// Data layout in HBM (one "level" of the bisection recursion):
//   * All subgraphs ("segments") of a level live in one block-diagonal graph of
//     N rows; segment s owns the contiguous rows [row0, row0 + n).
//   * The graph is stored as sliced ELL with slice height 32 (SELL-32): row r
//     sits in slice r >> 5 at lane r & 31, entry k of the row at
//     ent[slice_ptr[slice] + 32 k + lane].  An entry packs the column in its
//     low 29 bits and the integer weight (1..7, 0 = padding) in the top 3 bits,
//     so one 4-byte coalesced load per entry and warp gives both.  The
//     diagonal is never stored: the Laplacian action is
//     y_r = sum_k w_rk (x_r - x_{c_k}) (paper §4, L = D - A).
//   * Vectors are dense arrays over the level's N rows; a Lanczos basis is m+1
//     such arrays back to back.
//   * A "unit" is one Fiedler problem: the rows of a segment, or only the
//     rows of one of its connected components (masked by component key).
//   * Kernels run one CTA per "tile": a contiguous row range of one unit, so
//     every CTA reduces into exactly one unit.  The tiling of a unit depends
//     only on its row count, which makes every reduction's summation order —
//     and hence every result — independent of what else is in the batch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "rsb.h"
#include "rsb_test.h"

#define RSB_BLOCK 256
#define RSB_WARPS (RSB_BLOCK / 32)
#define RSB_MAXM 40                       // Krylov steps per cycle
#define RSB_MAXD 2                        // deflation vectors (cluster dim 3)
#define RSB_MAXC (1 + RSB_MAXD + RSB_MAXM)  // Gram-Schmidt coefficients
#define RSB_MAXKEEP 16                    // Ritz vectors kept by a thick restart
#define RSB_SSTRIDE (2 * RSB_MAXM * RSB_MAXM)  // doubles of S and Y per unit
#define RSB_MAXTILES_PER_UNIT 1024
#define RSB_MINR 2    // minimum rows per thread of a tile
// Tiles of a large level: rows per thread grow until the level has about this
// many tiles (eight waves of two CTAs on each of 152 SMs), so that a streaming
// kernel's tile spans many bulk-copy chunks and its pipeline fills
#define RSB_TARGET_TILES 2432
#define RSB_SUBR 4    // rows per thread handled between two CTA barriers
#define RSB_COLBITS 29
#define RSB_COLMASK 0x1FFFFFFFu
#define RSB_MAXN (1 << RSB_COLBITS)

// unit status
#define U_ACTIVE 0
#define U_CONVERGED 1
#define U_CAPPED 2
#define U_IDLE 3

// ----------------------------------------------------------------------------
// per-unit state (device)
// ----------------------------------------------------------------------------
struct Unit {
  // geometry, set by the host
  int32_t row0, nrows;   // row range of the owning segment in the level
  int32_t seg;           // owning segment
  int32_t masked;        // rows belong only when ckey[row] == key
  uint64_t key;
  int64_t n;             // rows of the unit
  int64_t k;             // rows that go left (R7 count inside the unit)
  int32_t tile0, ntile;  // tiles of this unit
  int32_t valid;         // the unit exists at this level (n >= 2)
  // solver state
  double isn;            // 1 / sqrt(n)
  double dmax;           // largest weighted degree in the unit
  double tolabs;         // tol * dmax
  int32_t m;             // basis size of a cycle for this unit
  int32_t msteps;        // basis size reached this cycle (m, or fewer on breakdown)
  int32_t j0;            // first new step of the cycle (kept Ritz vectors before it)
  int32_t kk;            // Ritz vectors kept for the next cycle (0: explicit restart)
  int32_t broke;         // the cycle ended on an invariant subspace
  int32_t keep;          // thick-restart size requested
  int32_t status;
  int32_t cycles;
  int32_t maxcycles;
  int32_t nd;            // deflation vectors in use
  int32_t inner;         // CG iterations of the last outer step
  int32_t cg_done;
  int64_t inner_total;
  double theta, resid, ynorm2;
  double beta0;          // norm of the first new vector of the cycle (unnormalised)
  double th[RSB_MAXKEEP + 1];  // smallest Ritz values of the last cycle
  double alpha[RSB_MAXM];
  double beta[RSB_MAXM + 1];
  double c1[RSB_MAXC], c2[RSB_MAXC];
  double t[RSB_MAXM];
  double cp[1 + RSB_MAXD];
  // CG scalars (§7): FP64 recurrences in both precisions
  double rr, cg_alpha, cg_beta, bnorm;
  double fz_rz, fz_ro;          // flexible CG: z.r and z.r_old of the new z
  double dz_src, dz_z, dz_qz;   // delayed second pass: scales of src, z and q_j in step D3
  double cz[1 + RSB_MAXD];      // flexible CG: projection coefficients of z
  double rq, lnorm2;
  // select / split
  double vmax, vmin, amax;
  double sign;
  double vk, tau;
  uint64_t sel_prefix;
  int64_t sel_k, sel_below, sel_eq;
  int64_t gstar;
  double gstar_v;
  int64_t below;
  int64_t cut[3];
  double lam[3];         // eigenvalue of each candidate solve
  double res[3];         // final residual of each candidate solve
  int32_t best;
  int32_t ncand;
  unsigned int cnt;      // last-CTA counter of the segmented reductions
  int32_t axis;          // RCB: coordinate axis of the split
};

struct Tile {
  int32_t unit;
  int32_t row0, row1;
  int32_t pad;
};

// ----------------------------------------------------------------------------
// device helpers
// ----------------------------------------------------------------------------
#ifdef __CUDACC__

__device__ __forceinline__ uint32_t ent_col(uint32_t e) { return e & RSB_COLMASK; }
__device__ __forceinline__ uint32_t ent_w(uint32_t e) { return e >> RSB_COLBITS; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of one double per thread, deterministic; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sm) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) sm[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < RSB_WARPS; ++i) s += sm[i];
  }
  __syncthreads();
  return s;
}

// SplitMix64 (Steele, Lea & Flood 2014): output for state x.
__device__ __host__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Start-vector entry 2 u - 1, u = top 53 bits of SplitMix64(s_d ^ gid) / 2^53.
__device__ __forceinline__ double start_value(uint64_t sd, int64_t gid) {
  const uint64_t h = splitmix64(sd ^ (uint64_t)gid);
  return (double)(h >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

// Unsigned key whose order is the numeric order of doubles.
__device__ __forceinline__ uint64_t dkey(double v) {
  const uint64_t b = (uint64_t)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_inv(uint64_t k) {
  const uint64_t b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  return __longlong_as_double((long long)b);
}

// An entry's weight (0..7) as an exact double built with integer operations
// (2^e (1 + m 2^-e) for w = 2^e + m), so that the FP64 Laplacian spends one FP64
// instruction per entry: GB300 retires about two FP64 operations per SM cycle.
__device__ __forceinline__ double weight_f64(uint32_t w) {
  const int e = 31 - __clz((int)(w | 1u));
  const unsigned long long m = (unsigned long long)(w - (1u << e)) << (52 - e);
  const unsigned long long bits = ((unsigned long long)(1023 + e) << 52) | m;
  return __longlong_as_double(w ? (long long)bits : 0ll);
}

// Laplacian action of one row, y_r = sum_k w_rk (x_r - x_{c_k}) in entry order
// (the order every other form of the action uses, so the results are the same
// bit for bit), for x that no thread of the launch writes: the row's entries
// are loaded eight at a time and their gathers issued together through the
// read-only path, so each thread keeps up to eight gathers in flight.
// Entries past the row's width are neither loaded nor gathered.
// In FP64 the row is d_r x_r - sum_k w_rk x_{c_k} (d_r = sum of the weights,
// exact): one FMA per entry, with a rounding error of about 1e-16 d_r |x| that
// FP64 can afford; FP32 keeps the differences, which are exact for close
// values and avoid the cancellation on smooth vectors.
template <typename V>
__device__ __forceinline__ V spmv_row_ro(const int64_t* __restrict__ slice_ptr,
                                         const uint32_t* __restrict__ ent,
                                         const V* __restrict__ x, int r, V xr) {
  const int64_t base = slice_ptr[r >> 5];
  const int width = (int)((slice_ptr[(r >> 5) + 1] - base) >> 5);
  const uint32_t* e = ent + base + (r & 31);
  V acc = V(0);
  uint32_t dsum = 0;
  for (int k0 = 0; k0 < width; k0 += 8) {
    uint32_t p[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) p[i] = k0 + i < width ? __ldg(e + 32 * (k0 + i)) : 0u;
    V xv[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) xv[i] = k0 + i < width ? __ldg(x + ent_col(p[i])) : xr;
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (k0 + i < width) {
        if constexpr (sizeof(V) == 8) {
          acc = fma(weight_f64(ent_w(p[i])), xv[i], acc);
          dsum += ent_w(p[i]);
        } else {
          acc += V(ent_w(p[i])) * (xr - xv[i]);
        }
      }
  }
  if constexpr (sizeof(V) == 8) return fma((double)dsum, xr, -acc);
  return acc;
}

// Row membership in a unit.
__device__ __forceinline__ bool unit_has(const Unit& u, const uint64_t* ckey, int r) {
  return !u.masked || ckey[r] == u.key;
}

// Compensated accumulator: FP64 plain, FP32 Kahan (paper-independent
// precision scheme: FP32 terms, compensated FP32 sums, FP64 across threads).
template <typename V> struct Acc;
template <> struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double get() const { return s; }
};
template <> struct Acc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double get() const { return (double)s - (double)c; }
};


// Warp total of per-lane accumulators, valid in lane 0.  FP64: plain
// butterfly.  FP32: the lanes' Kahan states (value s - c) are merged in FP32
// by error-free TwoSum steps (s1 + s2 = S + e exactly; the merged state is
// S, c1 + c2 - e), and only lane 0 converts to FP64: on GB300 an FP64
// instruction costs a warp about 16 SM cycles, an FP32 one a fraction of one.
__device__ __forceinline__ double warp_total(const Acc<double>& a) { return warp_sum(a.s); }
__device__ __forceinline__ double warp_total(const Acc<float>& a) {
  float s = a.s, c = a.c;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
    const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
    const float S = __fadd_rn(s, s2);
    const float bb = __fsub_rn(S, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(S, bb)), __fsub_rn(s2, bb));
    c = __fsub_rn(__fadd_rn(c, c2), e);
    s = S;
  }
  return (threadIdx.x & 31) == 0 ? (double)s - (double)c : 0.0;
}

// Block total of per-thread accumulators (warp_total per warp, then the warps
// in order in FP64); result valid in thread 0.
template <typename V>
__device__ __forceinline__ double block_total(const Acc<V>& a, double* sm) {
  const double v = warp_total(a);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) sm[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < RSB_WARPS; ++i) s += sm[i];
  }
  __syncthreads();
  return s;
}

// Gram-Schmidt coefficients in the vector type, converted once per CTA:
// cv[0] = V(coef[0] / sqrt(n)) for u0, cv[k] = V(coef[k]) otherwise.
template <typename V, bool CO>
__device__ __forceinline__ void stage_coef(const double* coef, int nc, double isn, V* cv) {
  for (int k = threadIdx.x; k < nc; k += RSB_BLOCK) {
    const double c = CO ? __ldcg(coef + k) : coef[k];
    cv[k] = k == 0 ? V(c * isn) : V(c);
  }
  __syncthreads();
}

// Last-CTA election of a unit's segmented reduction: every CTA of the unit
// has stored its partials; the CTA that arrives last reduces them in tile
// order (so the result does not depend on which CTA is last) and resets the
// counter for the next kernel.  No CTA waits on another.
__device__ __forceinline__ bool last_cta(unsigned int* cnt, int ntile) {
  __shared__ int am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(cnt, 1u);
    am_last = (prev == (unsigned)(ntile - 1));
    if (am_last) *cnt = 0u;
  }
  __syncthreads();
  if (am_last) __threadfence();
  return am_last != 0;
}

// Grid-wide barrier of a cooperative (co-resident) launch: generation counter,
// thread 0 of each CTA arrives and waits.  The wait is bounded (4 s of the
// global timer); on timeout the error word is set and every CTA that reaches a
// barrier afterwards returns false, so the kernel ends instead of hanging.
struct GridBar {
  unsigned int count;
  unsigned int gen;
  int err;
  int pad;
};

// Test hook of the failure path (set by rsb_test_poison_barrier).
extern int g_rsb_poison_barrier;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Arrival is an acquire-release add on the counter (it publishes the CTA's
// writes, which the CTA barrier ordered before it, and observes those of the
// CTAs that arrived earlier); the last CTA resets the counter and releases the
// next generation; the others spin on an acquire load of the generation.
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool grid_sync(GridBar* b, unsigned nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile int* verr = &b->err;
    const unsigned g = ld_acquire(&b->gen);
    const unsigned arrived = atom_add_acq_rel(&b->count, 1u);
    if (arrived == nblocks - 1) {
      asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(&b->count), "r"(0u) : "memory");
      asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(&b->gen), "r"(1u) : "memory");
    } else {
      const unsigned long long t0 = global_ns();
      unsigned spins = 0;
      while (ld_acquire(&b->gen) == g) {
        if (*verr) break;
        ++spins;
        if ((spins & 255u) == 0 && global_ns() - t0 > 4000000000ull) {
          atomicExch(&b->err, 1);
          break;
        }
        if (spins > 32) __nanosleep(32);
      }
    }
    s_ok = (*verr == 0);
  }
  __syncthreads();
  return s_ok != 0;
}

// Loads of data another CTA may have written earlier in the same launch go
// through L2 (L1 is not coherent across SMs).
template <bool CO, typename T>
__device__ __forceinline__ T ldc(const T* p) {
  if constexpr (CO) return __ldcg(p);
  else return *p;
}

// out[c] = sum_t partials[c * stride + t0 + t], t in [0, nt), c in [0, nc);
// fixed order, executed by the whole CTA.  Warp w owns coefficients w, w + 8,
// ...; eight lanes share a coefficient (four coefficients per warp at a
// time): lane s of a group adds tiles s, s + 8, ... (loads issued four at a
// time), then a three-level butterfly.  The FP64 adds are the cost on GB300
// (one FP64 warp instruction per ~64 cycles of an SM sub-partition), so no
// coefficient takes a 32-lane butterfly and unused coefficient slots cost
// nothing.
__device__ __forceinline__ void final_reduce(const double* partials, long long stride, int t0,
                                             int nt, int nc, double* out) {
  constexpr int CW = (RSB_MAXC + RSB_WARPS - 1) / RSB_WARPS;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 3, s = lane & 7;
  for (int pass = 0; pass < CW; pass += 4) {
    if (w + RSB_WARPS * pass >= nc) break;  // no coefficient of this warp is left
    const int c = w + RSB_WARPS * (pass + g);
    const bool on = pass + g < CW && c < nc;
    double acc = 0.0;
    if (on) {
      const double* p = partials + (long long)c * stride + t0;
      int t = s;
      for (; t + 24 < nt; t += 32) {
        const double a0 = __ldcg(p + t), a1 = __ldcg(p + t + 8);
        const double a2 = __ldcg(p + t + 16), a3 = __ldcg(p + t + 24);
        acc += (a0 + a1) + (a2 + a3);
      }
      for (; t < nt; t += 8) acc += __ldcg(p + t);
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 4);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    if (on && s == 0) out[c] = acc;
  }
  __syncthreads();
}

// ----------------------------------------------------------------------------
// mbarrier and 1-D bulk copies (cp.async.bulk global -> shared, completion
// counted in bytes on an mbarrier); every wait is bounded by the global timer
// ----------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity,
                                                  unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// All threads: wait for chunk ci (buffer ci & 1); false (uniform) when the
// copies did not complete in time, after flagging the grid error word and
// draining this CTA's copies still in flight (chunks ci and ci + 1).
__device__ __forceinline__ bool bulk_wait_chunk(uint64_t* bar, int ci, int nchunk, GridBar* gb) {
  const bool ok = mbar_wait_bounded(&bar[ci & 1], (ci >> 1) & 1, 2000000000ull);
  if (!__syncthreads_or(!ok)) return true;
  if (threadIdx.x == 0) {
    atomicMax(&gb->err, 1);
    // drain this CTA's copies still in flight before the CTA exits; if even
    // that runs out, the error word says so (2) and the call reports it
    bool drained = mbar_wait_bounded(&bar[ci & 1], (ci >> 1) & 1, 1000000000ull);
    if (ci + 1 < nchunk)
      drained = mbar_wait_bounded(&bar[(ci + 1) & 1], ((ci + 1) >> 1) & 1, 1000000000ull) &&
                drained;
    if (!drained) atomicMax(&gb->err, 2);
  }
  __syncthreads();
  return false;
}

#endif  // __CUDACC__

// ----------------------------------------------------------------------------
// host-side workspace
// ----------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

// Level-resident graph.
struct LevelGraph {
  int32_t n = 0;
  int64_t nslices = 0;
  int64_t* slice_ptr = nullptr;  // nslices + 1
  uint32_t* ent = nullptr;       // packed entries
  int32_t* deg = nullptr;        // weighted degree per row
  int64_t* gid = nullptr;
  int64_t* home = nullptr;       // index into the caller's (concatenated) output
  int32_t* row_seg = nullptr;
  int64_t nent = 0;
};

struct SegHost {
  int64_t row0, n;
  int32_t p0, p1, mesh;
  int64_t nleft;
};

// Error helpers (host)
int rsb_set_cuda_error(cudaError_t e, const char* where);
int rsb_set_error(int code, const std::string& what);
void rsb_count_launch(int k = 1);

// Kernel timing (rsb_profile_begin/end): families of include/rsb.h.
enum {
  PROF_NONE = 0, PROF_LZ_A = 1, PROF_LZ_B = 2, PROF_LZ_C = 3, PROF_CG_AP = 4, PROF_SPMV = 5,
  PROF_CYCLE = 6, PROF_LZ_A2 = 7, PROF_AMG = 8, PROF_NFAM = 9
};
int prof_before(int family, cudaStream_t s);      // event pair index or -1
void prof_after(int idx, cudaStream_t s);
void prof_collect();                              // after a stream sync
void prof_capture_begin();
std::vector<int> prof_capture_end();              // pairs recorded during a capture
void prof_replay(const std::vector<int>& pairs);  // a graph holding them was launched
unsigned long long* prof_bytes(int family);       // device byte counter or nullptr

#define RSB_CK(call)                                              \
  do {                                                            \
    cudaError_t e__ = (call);                                     \
    if (e__ != cudaSuccess) return rsb_set_cuda_error(e__, #call); \
  } while (0)
#define RSB_CKL(where)                                                         \
  do {                                                                         \
    rsb_count_launch();                                                        \
    cudaError_t e__ = cudaGetLastError();                                      \
    if (e__ != cudaSuccess) return rsb_set_cuda_error(e__, where);             \
  } while (0)

// Grow-only device buffer.
int devbuf_reserve(DevBuf& b, size_t bytes);
template <typename T>
static inline T* dptr(DevBuf& b) {
  return reinterpret_cast<T*>(b.p);
}

// ----------------------------------------------------------------------------
// launchers (graph.cu); the others are declared where they are used
// ----------------------------------------------------------------------------
int launch_validate(const int64_t* row_ptr, const int32_t* col, const int32_t* wt, int64_t n,
                    int symmetric, int* flag, cudaStream_t s);
int launch_row_lengths(const int64_t* row_ptr, int64_t n, int32_t* len, cudaStream_t s,
                       const int64_t* perm = nullptr);
int launch_slice_widths(const int32_t* len, int64_t n, int64_t* slice_sz, cudaStream_t s);
int launch_fill_sell(const int64_t* row_ptr, const int32_t* col, const int32_t* wt,
                     const int64_t* gid_in, int64_t n, int64_t row_off, int64_t home_off,
                     int32_t seg, const int64_t* slice_ptr, uint32_t* ent, int32_t* deg,
                     int64_t* gid, int64_t* home, int32_t* row_seg, cudaStream_t s,
                     const int64_t* perm = nullptr, const int32_t* iperm = nullptr);
int launch_rcb_vector(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units,
                      const double* coords, double* v, double* partials, cudaStream_t s);
int launch_scan_i64(const int64_t* in, int64_t* out_excl, int64_t n, void* tmp, size_t tmp_bytes,
                    cudaStream_t s);
size_t scan_tmp_bytes(int64_t n);
int launch_spmv_f64(const LevelGraph& G, const double* x, double* y, cudaStream_t s);
int launch_spmv_f32(const LevelGraph& G, const float* x, float* y, cudaStream_t s);
int launch_cc(const LevelGraph& G, int32_t* parent, uint64_t* ckey, int* flag, cudaStream_t s);
int launch_comp_count(const LevelGraph& G, const int32_t* parent, int32_t* seg_ncomp,
                      cudaStream_t s);
int launch_compact(const LevelGraph& G, LevelGraph& H, const uint8_t* side,
                   const int64_t* seg_row0_old, const int64_t* seg_nleft,
                   const int32_t* seg_child0, int32_t nseg, int64_t* newpos, int64_t* tmp64,
                   int32_t* len, int64_t* slice_sz, void* scan_tmp, size_t scan_tmp_bytes,
                   DevBuf& ent_buf, cudaStream_t s);
int launch_write_parts(const LevelGraph& G, const int32_t* seg_p0, int32_t* part_concat,
                       cudaStream_t s);
int launch_degree_max(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units,
                      const uint64_t* ckey, double* partials, cudaStream_t s);
int launch_split_assign(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units,
                        const uint64_t* ckey, const double* v, uint8_t* side, int cand,
                        cudaStream_t s);

// solver buffers of one precision (V = double or float)
struct SolveBufs {
  void* Q = nullptr;       // M x N basis vectors
  void* W0 = nullptr;      // work vectors
  void* W1 = nullptr;
  void* Y = nullptr;
  void* X = nullptr;       // CG
  void* R = nullptr;
  void* P = nullptr;
  void* AP = nullptr;
  const double* D[RSB_MAXD] = {nullptr, nullptr};  // deflation vectors (FP64)
  double* partials = nullptr;
  int* n_active = nullptr;       // device: units still iterating
  int* n_cg = nullptr;           // device: units whose CG still runs
  long long* stat_cycles = nullptr;
  int* h_active = nullptr;       // pinned host word for read-backs
  struct GridBar* gb = nullptr;  // barrier of the persistent cycle kernel
  double* S = nullptr;           // per-unit projected matrices and Ritz vectors
  int* jmin = nullptr;           // device: smallest next-cycle start step (2 slots)
  void* Z0 = nullptr;            // block Lanczos: interleaved residual blocks (4 values/row)
  void* Z1 = nullptr;
  void* bu = nullptr;            // block Lanczos: per-unit block state
  int64_t N = 0;
  int trmax = 0;                 // largest tile of the level, rows
  int maxcycles = 0;             // cycle cap of the current solve
};
