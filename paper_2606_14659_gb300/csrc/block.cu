// block.cu — thick-restarted block Lanczos for the Fiedler vector, batched
// over all units of a level (the block extension §9 names for a nearly
// repeated lambda_2; the single-vector method of §6 is in solver.cu).
//
// A unit's basis holds up to m = krylov_dim columns q_0..q_{m-1}.  A block
// step at column j (the columns j..j+B-1 are new) runs four launches:
//   spmm: Q_new = W R^-1 (W: the residual block, R: its Cholesky factor) into
//         q_j..q_{j+B-1}, and Z = L Q_new = (L W) R^-1, one pass over the
//         sliced-ELL graph for all B vectors (W is stored interleaved, so one
//         vector load per neighbour serves every column);
//   dots: first Gram-Schmidt pass coefficients C1 = [1/sqrt(n), D, q_0..]^T Z;
//   bt:   Z -= [..] C1 and the second pass's coefficients C2; columns j..j+B-1
//         of the projected matrix S = Q^T L Q are C1 + C2 on the basis;
//   c:    Z -= [..] C2 and the Gram matrix Z^T Z, whose Cholesky factor (taken
//         on the correlation matrix, so columns of very different norms are
//         fine) normalises the next block; nearly dependent columns end the
//         unit's cycle.
// dots, bt and c stage the basis rows of a 256-row chunk and the chunk of Z in
// shared memory with bulk copies (cp.async.bulk on an mbarrier, double
// buffered), so every basis vector is read from DRAM once per launch for all B
// columns.  A cycle ends with the Ritz pairs of S (the Jacobi solver of
// solver.cu), the Ritz vector y = Q s_1, the thick-restart basis q_i = Q s_i
// (i < kk) in place and the true residual ||L y - theta y||.  kk = keep +
// ((m - keep) mod B) so that whole blocks fill the basis again.  The start
// block (and the explicit restart after a breakdown: y and fresh columns) is
// projected by the same dots/bt/c launches against the fixed basis alone.
//
// Precision as in solver.cu: V = float keeps the vectors, SpMM and updates in
// FP32 with compensated per-thread sums; every cross-thread sum, coefficient,
// S entry, Gram matrix and Cholesky factor is FP64.
#include <algorithm>

#include "rsb_internal.cuh"

#define RSB_MAXB 4
#define BZ 4                           // stride of an interleaved block row
#define BSLOTS (RSB_MAXC * RSB_MAXB)   // coefficient slots of one pass
#define MAXCW ((RSB_MAXC + RSB_WARPS - 1) / RSB_WARPS)

struct BlkUnit {
  double c1[BSLOTS];  // first-pass coefficients, slot c * B + b
  double c2[BSLOTS];  // second-pass coefficients
  double rinv[RSB_MAXB * RSB_MAXB];  // R^-1 of the residual block, row-major
  int pending;        // the start block must be built and projected
  int pad[3];
};

template <typename V>
struct BlkArgs {
  const int64_t* slice_ptr;
  const uint32_t* ent;
  const int64_t* gid;
  const Tile* tiles;
  Unit* units;
  BlkUnit* bu;
  const uint64_t* ckey;
  V* Q;
  long long N;  // basis stride
  V* Z0;        // interleaved blocks, BZ values per row
  V* Z1;
  V* Y;
  const double* D0;
  const double* D1;
  double* partials;
  long long stride;
  int* n_active;
  long long* stat_cycles;
  double* S;
  uint64_t seedbase;  // seed + deflation count
  GridBar* gb;
  unsigned long long* pb_a;  // profiling byte counters (nullptr when off)
  unsigned long long* pb_a2;
  unsigned long long* pb_b;
  unsigned long long* pb_c;
};

__device__ __forceinline__ double* unit_Sb(double* S, int ui) {
  return S + (long long)ui * RSB_SSTRIDE;
}

// Block step t of the cycle for unit u (t < 0: the start block).  Returns the
// first new column j, or -1 when the unit does not take part.
template <int B>
__device__ __forceinline__ int blk_col(const Unit& u, const BlkUnit& b, int t) {
  if (__ldcg(&u.status) != U_ACTIVE) return -1;
  if (t < 0) return __ldcg(&b.pending) ? 0 : -1;
  if (__ldcg(&b.pending)) return -1;
  const int j = __ldcg(&u.j0) + t * B;
  return j + B <= __ldcg(&u.msteps) ? j : -1;
}

// out[c] = sum over the unit's tiles of partials[c * stride + tile], c < nc,
// fixed order (as final_reduce, for up to BSLOTS coefficients).
__device__ __forceinline__ void final_reduce_b(const double* partials, long long stride, int t0,
                                               int nt, int nc, double* out) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 3, s = lane & 7;
  for (int base = 0; base < nc; base += 4 * RSB_WARPS) {
    const int c = base + w * 4 + g;
    double acc = 0.0;
    if (c < nc) {
      const double* p = partials + (long long)c * stride + t0;
      int tt = s;
      for (; tt + 24 < nt; tt += 32) {
        const double a0 = __ldcg(p + tt), a1 = __ldcg(p + tt + 8);
        const double a2 = __ldcg(p + tt + 16), a3 = __ldcg(p + tt + 24);
        acc += (a0 + a1) + (a2 + a3);
      }
      for (; tt < nt; tt += 8) acc += __ldcg(p + tt);
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 4);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    if (c < nc && s == 0) out[c] = acc;
  }
  __syncthreads();
}

// ----------------------------------------------------------------------------
// chunk staging: rows [c0, c1) of q_0..q_{nq-1} (rounded out to 16 bytes) and
// of the interleaved block Z into buffer b; thread 0 only
// ----------------------------------------------------------------------------
template <typename V>
struct BStage {
  static constexpr int AL = 16 / sizeof(V);   // rows per 16 bytes of a basis vector
  static constexpr int CRB = RSB_BLOCK + AL;  // staged rows per basis vector
  static constexpr int ZR = RSB_BLOCK * BZ;   // staged values of the Z chunk
  static size_t bytes(int nq) { return 2 * ((size_t)nq * CRB + ZR) * sizeof(V); }
};

template <typename V>
__device__ __forceinline__ void stage_issue(const BlkArgs<V>& a, const V* Zc, V* buf,
                                            uint64_t* bar, int nq, int b, int c0, int c1) {
  constexpr int AL = BStage<V>::AL, CRB = BStage<V>::CRB, ZR = BStage<V>::ZR;
  const int a0 = c0 & ~(AL - 1);
  const int len = (c1 - a0 + AL - 1) / AL * AL;
  const unsigned qbytes = (unsigned)(len * sizeof(V));
  const unsigned zbytes = (unsigned)((c1 - c0) * BZ * sizeof(V));
  V* dst = buf + (size_t)b * ((size_t)nq * CRB + ZR);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_expect_tx(&bar[b], qbytes * (unsigned)nq + zbytes);
  for (int k = 0; k < nq; ++k)
    bulk_g2s(dst + (size_t)k * CRB, a.Q + (long long)k * a.N + a0, qbytes, &bar[b]);
  bulk_g2s(dst + (size_t)nq * CRB, Zc + (long long)c0 * BZ, zbytes, &bar[b]);
}

// Coefficients of pass `pass` (0: c1, 1: c2) in the vector type:
// cv[c * B + b], with the u0 coefficient already times 1/sqrt(n).
template <typename V, int B>
__device__ __forceinline__ void stage_coef_b(const double* coef, int nc, double isn, V* cv) {
  for (int k = threadIdx.x; k < nc * B; k += RSB_BLOCK) {
    const double c = __ldcg(coef + k);
    cv[k] = k < B ? V(c * isn) : V(c);
  }
  __syncthreads();
}

// z[b] -= sum_c cv[c][b] basis_c[row] for one row (basis: 1 on unit rows, D,
// q_0..q_{nq-1} staged at Qc[k * CRB + rl])
template <typename V, int B>
__device__ __forceinline__ void upd_row(const BlkArgs<V>& a, const V* cv, int nd, int nq,
                                        const V* Qc, int rl, int r, bool in_unit, V (&z)[B]) {
  constexpr int CRB = BStage<V>::CRB;
  if (in_unit)
#pragma unroll
    for (int b = 0; b < B; ++b) z[b] -= cv[b];
  for (int l = 0; l < nd; ++l) {
    const V d = V((l == 0 ? a.D0 : a.D1)[r]);
#pragma unroll
    for (int b = 0; b < B; ++b) z[b] -= cv[(1 + l) * B + b] * d;
  }
  const V* cq = cv + (1 + nd) * B;
  for (int k = 0; k < nq; ++k) {
    const V q = Qc[(size_t)k * CRB + rl];
#pragma unroll
    for (int b = 0; b < B; ++b) z[b] -= cq[k * B + b] * q;
  }
}

// Dots of [1, D, q_0..q_{nq-1}] with the staged chunk Zs (nr rows): warp w
// owns coefficients w, w + 8, ...; lanes walk the rows.
template <typename V, int B>
__device__ __forceinline__ void chunk_dots(const BlkArgs<V>& a, int nd, int nc, const V* Qc,
                                           const V* Zs, int c0, int nr, Acc<V> (&acc)[MAXCW][B]) {
  constexpr int CRB = BStage<V>::CRB;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < MAXCW; ++i) {
    const int c = w + RSB_WARPS * i;
    if (c >= nc) continue;
    for (int rl = lane; rl < nr; rl += 32) {
      V q;
      if (c == 0) q = V(1);
      else if (c <= nd) q = V((c == 1 ? a.D0 : a.D1)[c0 + rl]);
      else q = Qc[(size_t)(c - 1 - nd) * CRB + rl];
#pragma unroll
      for (int b = 0; b < B; ++b) acc[i][b].add(q * Zs[rl * BZ + b]);
    }
  }
}

template <typename V, int B>
__device__ __forceinline__ void store_dots_b(const BlkArgs<V>& a, int nc, Acc<V> (&acc)[MAXCW][B],
                                             int tix) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < MAXCW; ++i) {
    const int c = w + RSB_WARPS * i;
    if (c >= nc) continue;
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const double s = warp_total(acc[i][b]);
      if (lane == 0) a.partials[(long long)(c * B + b) * a.stride + tix] = s;
    }
  }
}

// ----------------------------------------------------------------------------
// start block: column c = start vector of seed (seedbase + (c + B * cycles) << 32)
// on unit rows (column 0 = y after a breakdown restart), interleaved into Z0
// ----------------------------------------------------------------------------
template <typename V, int B>
__global__ void __launch_bounds__(RSB_BLOCK) k_blk_start(BlkArgs<V> a) {
  const Tile t = a.tiles[blockIdx.x];
  const Unit& u = a.units[t.unit];
  if (blk_col<B>(u, a.bu[t.unit], -1) < 0) return;
  const int cyc = u.cycles;
  uint64_t sd[B];
#pragma unroll
  for (int b = 0; b < B; ++b)
    sd[b] = splitmix64(a.seedbase + ((uint64_t)(b + B * cyc) << 32));
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    const bool in = unit_has(u, a.ckey, r);
    V z[BZ];
#pragma unroll
    for (int b = 0; b < BZ; ++b) z[b] = V(0);
    if (in) {
#pragma unroll
      for (int b = 0; b < B; ++b)
        z[b] = (b == 0 && cyc > 0) ? a.Y[r] : V(start_value(sd[b], a.gid[r]));
    }
#pragma unroll
    for (int b = 0; b < BZ; ++b) a.Z0[(long long)r * BZ + b] = z[b];
  }
}

// ----------------------------------------------------------------------------
// spmm: Q_new = W R^-1 into q_j..q_{j+B-1}; Z = (L W) R^-1
// ----------------------------------------------------------------------------
template <typename V, int B>
__global__ void __launch_bounds__(RSB_BLOCK) k_blk_spmm(BlkArgs<V> a, int t) {
  __shared__ V ri[RSB_MAXB * RSB_MAXB];
  const Tile tl = a.tiles[blockIdx.x];
  const Unit& u = a.units[tl.unit];
  const int j = blk_col<B>(u, a.bu[tl.unit], t);
  if (j < 0) return;
  if (threadIdx.x < B * B) ri[threadIdx.x] = V(__ldcg(&a.bu[tl.unit].rinv[threadIdx.x]));
  __syncthreads();
  const V* W = (t & 1) ? a.Z1 : a.Z0;
  V* Zo = (t & 1) ? a.Z0 : a.Z1;
  unsigned long long pbytes = 0;
  for (int r = tl.row0 + threadIdx.x; r < tl.row1; r += RSB_BLOCK) {
    V wr[BZ];
    if constexpr (sizeof(V) == 4) {
      const float4 v = __ldcg(reinterpret_cast<const float4*>(W) + r);
      wr[0] = v.x; wr[1] = v.y; wr[2] = v.z; wr[3] = v.w;
    } else {
#pragma unroll
      for (int b = 0; b < BZ; ++b) wr[b] = __ldcg(W + (long long)r * BZ + b);
    }
    const int64_t base = a.slice_ptr[r >> 5];
    const int width = (int)((a.slice_ptr[(r >> 5) + 1] - base) >> 5);
    const uint32_t* e = a.ent + base + (r & 31);
    V acc[B];
#pragma unroll
    for (int b = 0; b < B; ++b) acc[b] = V(0);
#pragma unroll 4
    for (int k = 0; k < width; ++k) {
      const uint32_t p = __ldg(e + 32 * k);
      const V wgt = V(ent_w(p));
      const long long c = ent_col(p);
      if constexpr (sizeof(V) == 4) {
        const float4 x = __ldg(reinterpret_cast<const float4*>(W) + c);
        const V xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int b = 0; b < B; ++b) acc[b] += wgt * (wr[b] - xs[b]);
      } else {
#pragma unroll
        for (int b = 0; b < B; ++b) acc[b] += wgt * (wr[b] - __ldg(W + c * BZ + b));
      }
    }
    V zo[BZ];
#pragma unroll
    for (int b = 0; b < BZ; ++b) zo[b] = V(0);
#pragma unroll
    for (int i = 0; i < B; ++i) {
      V q = V(0), z = V(0);
#pragma unroll
      for (int l = 0; l <= i; ++l) {
        q += wr[l] * ri[l * B + i];
        z += acc[l] * ri[l * B + i];
      }
      a.Q[(long long)(j + i) * a.N + r] = q;
      zo[i] = z;
    }
    if constexpr (sizeof(V) == 4) {
      reinterpret_cast<float4*>(Zo)[r] = make_float4(zo[0], zo[1], zo[2], zo[3]);
    } else {
#pragma unroll
      for (int b = 0; b < BZ; ++b) Zo[(long long)r * BZ + b] = zo[b];
    }
    if (a.pb_a) pbytes += 4ull * width + sizeof(V) * (unsigned long long)(2 * BZ + B);
  }
  if (a.pb_a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pbytes += __shfl_xor_sync(0xffffffffu, pbytes, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(a.pb_a, pbytes);
  }
}

// ----------------------------------------------------------------------------
// The three Gram-Schmidt launches share one chunk loop: stage the chunk's rows
// of q_0..q_{nq-1} and of Z, then (mode 0) dots only, (mode 1) update with c1
// then dots, (mode 2) update with c2 then the Gram matrix.
// ----------------------------------------------------------------------------
template <typename V, int B, int MODE>
__global__ void __launch_bounds__(RSB_BLOCK, 2) k_blk_gs(BlkArgs<V> a, int t) {
  extern __shared__ __align__(128) unsigned char bsh[];
  constexpr int AL = BStage<V>::AL, CRB = BStage<V>::CRB, ZR = BStage<V>::ZR;
  constexpr int NG = B * (B + 1) / 2;
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ V cv[BSLOTS];
  __shared__ double out[BSLOTS];
  __shared__ double sm[RSB_WARPS];
  const int tix = blockIdx.x;
  const Tile tl = a.tiles[tix];
  Unit& u = a.units[tl.unit];
  BlkUnit& bu = a.bu[tl.unit];
  const int j = blk_col<B>(u, bu, t);
  if (j < 0) return;
  const int nd = u.nd;
  const int nq = t < 0 ? 0 : j + B;
  const int nc = 1 + nd + nq;
  V* Zc = t < 0 ? a.Z0 : ((t & 1) ? a.Z0 : a.Z1);
  V* buf = reinterpret_cast<V*>(bsh);
  const int nchunk = (tl.row1 - tl.row0 + RSB_BLOCK - 1) / RSB_BLOCK;
  const bool masked = u.masked;
  const uint64_t key = u.key;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (MODE == 1) stage_coef_b<V, B>(bu.c1, nc, u.isn, cv);
  if (MODE == 2) stage_coef_b<V, B>(bu.c2, nc, u.isn, cv);
  __syncthreads();
  if (threadIdx.x == 0)
    stage_issue(a, Zc, buf, bar, nq, 0, tl.row0, min(tl.row1, tl.row0 + RSB_BLOCK));
  Acc<V> acc[MAXCW][B];
  Acc<V> gacc[NG];
  unsigned long long pbytes = 0;
  for (int ci = 0; ci < nchunk; ++ci) {
    if (threadIdx.x == 0 && ci + 1 < nchunk) {
      const int n0 = tl.row0 + (ci + 1) * RSB_BLOCK;
      stage_issue(a, Zc, buf, bar, nq, (ci + 1) & 1, n0, min(tl.row1, n0 + RSB_BLOCK));
    }
    if (!bulk_wait_chunk(bar, ci, nchunk, a.gb)) return;
    const int c0 = tl.row0 + ci * RSB_BLOCK;
    const int c1 = min(tl.row1, c0 + RSB_BLOCK);
    const int nr = c1 - c0;
    V* bb = buf + (size_t)(ci & 1) * ((size_t)nq * CRB + ZR);
    const V* Qc = bb + (c0 - (c0 & ~(AL - 1)));
    V* Zs = bb + (size_t)nq * CRB;
    if (MODE > 0) {
      const int rl = threadIdx.x;
      if (rl < nr) {
        const int r = c0 + rl;
        V z[B];
#pragma unroll
        for (int b = 0; b < B; ++b) z[b] = Zs[rl * BZ + b];
        const bool in_unit = !masked || a.ckey[r] == key;
        upd_row<V, B>(a, cv, nd, nq, Qc, rl, r, in_unit, z);
#pragma unroll
        for (int b = 0; b < B; ++b) {
          Zs[rl * BZ + b] = z[b];
          Zc[(long long)r * BZ + b] = z[b];
        }
        if (MODE == 2) {
          int g = 0;
#pragma unroll
          for (int b1 = 0; b1 < B; ++b1)
#pragma unroll
            for (int b2 = b1; b2 < B; ++b2) gacc[g++].add(z[b1] * z[b2]);
        }
      }
      __syncthreads();
    }
    if (MODE < 2) chunk_dots<V, B>(a, nd, nc, Qc, Zs, c0, nr, acc);
    if (a.pb_a2 || a.pb_b || a.pb_c)
      if ((int)threadIdx.x < nr)
        pbytes += sizeof(V) * (unsigned long long)(nq + (MODE > 0 ? 2 * BZ : BZ)) + 8ull * nd;
    __syncthreads();
  }
  unsigned long long* pb = MODE == 0 ? a.pb_a2 : (MODE == 1 ? a.pb_b : a.pb_c);
  if (pb) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pbytes += __shfl_xor_sync(0xffffffffu, pbytes, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(pb, pbytes);
  }
  if (MODE < 2) {
    store_dots_b<V, B>(a, nc, acc, tix);
  } else {
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const double s = block_total(gacc[g], sm);
      if (threadIdx.x == 0) a.partials[(long long)g * a.stride + tix] = s;
    }
  }
  if (!last_cta(&u.cnt, u.ntile)) return;
  if (MODE < 2) {
    final_reduce_b(a.partials, a.stride, u.tile0, u.ntile, nc * B, out);
    double* dst = MODE == 0 ? bu.c1 : bu.c2;
    for (int k = threadIdx.x; k < nc * B; k += RSB_BLOCK) dst[k] = k < B ? out[k] * u.isn : out[k];
    __syncthreads();
    if (MODE == 1 && t >= 0) {
      // columns j..j+B-1 of S: c1 + c2 on q_0..q_{j+B-1}, the diagonal block symmetrised
      double* Sm = unit_Sb(a.S, tl.unit);
      const int off = (1 + nd) * B;
      for (int idx = threadIdx.x; idx < (j + B) * B; idx += RSB_BLOCK) {
        const int k = idx / B, b = idx % B;
        double v = __ldcg(&bu.c1[off + idx]) + out[off + idx];
        if (k >= j) {
          const int kb = k - j;
          const int mirror = off + (j + b) * B + kb;
          v = 0.5 * (v + __ldcg(&bu.c1[mirror]) + out[mirror]);
        }
        Sm[k * RSB_MAXM + (j + b)] = v;
        Sm[(j + b) * RSB_MAXM + k] = v;
      }
    }
    return;
  }
  // MODE 2: Gram matrix -> Cholesky factor of the next block (FP64, thread 0)
  final_reduce_b(a.partials, a.stride, u.tile0, u.ntile, NG, out);
  if (threadIdx.x != 0) return;
  double G[B][B];
  {
    int g = 0;
    for (int b1 = 0; b1 < B; ++b1)
      for (int b2 = b1; b2 < B; ++b2) {
        G[b1][b2] = out[g];
        G[b2][b1] = out[g];
        ++g;
      }
  }
  const double tiny = 1e-14 * u.dmax;
  const double pivot_min = sizeof(V) == 4 ? 1e-4 : 1e-12;
  double dsc[B], L[B][B];
  bool ok = true;
  for (int b = 0; b < B; ++b) {
    dsc[b] = sqrt(fmax(G[b][b], 0.0));
    ok = ok && dsc[b] > tiny;
  }
  for (int i = 0; ok && i < B; ++i) {
    for (int k = 0; k <= i; ++k) {
      double sum = G[i][k] / (dsc[i] * dsc[k]);
      for (int l = 0; l < k; ++l) sum -= L[i][l] * L[k][l];
      if (k == i) {
        if (sum < pivot_min) ok = false;
        else L[i][i] = sqrt(sum);
      } else {
        L[i][k] = sum / L[k][k];
      }
    }
  }
  if (!ok) {
    if (t >= 0) {  // the block after q_{j+B-1} cannot be formed: the cycle ends here
      u.msteps = j + B;
      u.broke = 1;
    } else {       // a start block without full rank (not expected): give up on the unit
      bu.pending = 0;
      u.status = U_CAPPED;
      atomicSub(a.n_active, 1);
    }
    return;
  }
  // R = Rs diag(dsc) with Rs = L^T; R^-1 = diag(1/dsc) Rs^-1 (upper triangular)
  double Li[B][B];  // inverse of the lower factor L
  for (int i = 0; i < B; ++i)
    for (int k = 0; k < B; ++k) Li[i][k] = 0.0;
  for (int i = 0; i < B; ++i) {
    Li[i][i] = 1.0 / L[i][i];
    for (int k = 0; k < i; ++k) {
      double sum = 0.0;
      for (int l = k; l < i; ++l) sum += L[i][l] * Li[l][k];
      Li[i][k] = -sum / L[i][i];
    }
  }
  // Rs^-1 = (L^-1)^T; R^-1[l][i] = Rs^-1[l][i] / dsc[l] = Li[i][l] / dsc[l]
  for (int l = 0; l < B; ++l)
    for (int i = 0; i < B; ++i) bu.rinv[l * B + i] = (i >= l) ? Li[i][l] / dsc[l] : 0.0;
  if (t < 0) bu.pending = 0;
}

// ----------------------------------------------------------------------------
// end of a cycle: Ritz vector and thick-restart basis, residual and decision
// ----------------------------------------------------------------------------
template <typename V, int B>
__global__ void __launch_bounds__(RSB_BLOCK) k_blk_ritz(BlkArgs<V> a) {
  const Tile t = a.tiles[blockIdx.x];
  const Unit& u = a.units[t.unit];
  if (u.status != U_ACTIVE) return;
  const int K = u.msteps;
  const int kk = u.kk;
  const int T = (K - u.j0) / B;  // block steps this cycle: the residual block is in Z[T & 1]
  const double* Ym = unit_Sb(a.S, t.unit) + RSB_MAXM * RSB_MAXM;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    V q[RSB_MAXM];
#pragma unroll
    for (int l = 0; l < RSB_MAXM; ++l) q[l] = l < K ? a.Q[(long long)l * a.N + r] : V(0);
    for (int i = 0; i <= kk; ++i) {
      V acc = V(0);
#pragma unroll
      for (int l = 0; l < RSB_MAXM; ++l)
        if (l < K) acc += V(Ym[l * RSB_MAXM + i]) * q[l];
      if (i == 0) a.Y[r] = acc;
      if (i < kk) a.Q[(long long)i * a.N + r] = acc;
    }
    if (kk > 0 && (T & 1))
#pragma unroll
      for (int b = 0; b < BZ; ++b) a.Z0[(long long)r * BZ + b] = a.Z1[(long long)r * BZ + b];
  }
  if (a.pb_c && threadIdx.x == 0)
    atomicAdd(a.pb_c, (unsigned long long)(t.row1 - t.row0) * sizeof(V) * (K + kk + 1));
}

template <typename V, int B>
__global__ void __launch_bounds__(RSB_BLOCK) k_blk_resid(BlkArgs<V> a) {
  __shared__ double sm[RSB_WARPS];
  __shared__ double out[2];
  const Tile t = a.tiles[blockIdx.x];
  Unit& u = a.units[t.unit];
  if (u.status != U_ACTIVE) return;
  const V th = V(u.theta);
  Acc<V> r2, y2;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    const V yr = a.Y[r];
    const int64_t base = a.slice_ptr[r >> 5];
    const int width = (int)((a.slice_ptr[(r >> 5) + 1] - base) >> 5);
    const uint32_t* e = a.ent + base + (r & 31);
    V ly = V(0);
#pragma unroll 4
    for (int k = 0; k < width; ++k) {
      const uint32_t p = __ldg(e + 32 * k);
      ly += V(ent_w(p)) * (yr - a.Y[ent_col(p)]);
    }
    const V res = ly - th * yr;
    r2.add(res * res);
    y2.add(yr * yr);
  }
  const double s0 = block_total(r2, sm);
  const double s1 = block_total(y2, sm);
  if (threadIdx.x == 0) {
    a.partials[blockIdx.x] = s0;
    a.partials[a.stride + blockIdx.x] = s1;
  }
  if (!last_cta(&u.cnt, u.ntile)) return;
  final_reduce_b(a.partials, a.stride, u.tile0, u.ntile, 2, out);
  if (threadIdx.x == 0) {
    u.ynorm2 = out[1];
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
      u.j0 = u.kk;  // thick restart: the kept Ritz vectors are q_0..q_{kk-1}
      u.msteps = u.kk + (u.m - u.kk) / B * B;
    } else {
      u.j0 = 0;     // explicit restart from y and fresh start columns
      u.msteps = u.m / B * B;
      a.bu[t.unit].pending = 1;
    }
    u.broke = 0;
  }
  __syncthreads();
  if (u.status == U_ACTIVE) {
    // next cycle's S = diag(kept Ritz values); explicit restarts clear it all
    double* Sm = unit_Sb(a.S, t.unit);
    const int kk = u.j0;
    for (int idx = threadIdx.x; idx < RSB_MAXM * RSB_MAXM; idx += RSB_BLOCK) {
      const int i = idx / RSB_MAXM, k = idx % RSB_MAXM;
      Sm[idx] = (i == k && i < kk) ? u.th[i] : 0.0;
    }
  }
}

// solve set-up of the units taking part: block state, first-cycle basis size
template <int B>
__global__ void k_blk_init(Unit* units, BlkUnit* bu, int nunits, int keep_b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nunits) return;
  Unit& u = units[i];
  if (u.status != U_ACTIVE) return;
  u.j0 = 0;
  u.msteps = u.m / B * B;
  u.keep = keep_b;
  u.kk = 0;
  u.broke = 0;
  bu[i].pending = 1;
}

// ----------------------------------------------------------------------------
// host driver
// ----------------------------------------------------------------------------
int launch_lz_eig(int f32, Unit* units, double* S, int nunits, cudaStream_t s);

template <typename V, int B>
static int blk_cycle(BlkArgs<V>& a, int ntiles, int nunits, int M, int keep_b, int f32,
                     cudaStream_t s) {
  const size_t sh_start = BStage<V>::bytes(0);
  const size_t sh_full = BStage<V>::bytes(M);
  // start block (units with a pending start only): build, then project twice
  k_blk_start<V, B><<<ntiles, RSB_BLOCK, 0, s>>>(a);
  RSB_CKL("k_blk_start");
  k_blk_gs<V, B, 0><<<ntiles, RSB_BLOCK, sh_start, s>>>(a, -1);
  RSB_CKL("k_blk_gs<0>(start)");
  k_blk_gs<V, B, 1><<<ntiles, RSB_BLOCK, sh_start, s>>>(a, -1);
  RSB_CKL("k_blk_gs<1>(start)");
  k_blk_gs<V, B, 2><<<ntiles, RSB_BLOCK, sh_start, s>>>(a, -1);
  RSB_CKL("k_blk_gs<2>(start)");
  const int T = M / B;
  for (int t = 0; t < T; ++t) {
    const size_t sh = BStage<V>::bytes(std::min(M, (t + 1) * B + keep_b));
    int pi = prof_before(PROF_LZ_A, s);
    k_blk_spmm<V, B><<<ntiles, RSB_BLOCK, 0, s>>>(a, t);
    RSB_CKL("k_blk_spmm");
    prof_after(pi, s);
    pi = prof_before(PROF_LZ_A2, s);
    k_blk_gs<V, B, 0><<<ntiles, RSB_BLOCK, sh, s>>>(a, t);
    RSB_CKL("k_blk_gs<0>");
    prof_after(pi, s);
    pi = prof_before(PROF_LZ_B, s);
    k_blk_gs<V, B, 1><<<ntiles, RSB_BLOCK, sh, s>>>(a, t);
    RSB_CKL("k_blk_gs<1>");
    prof_after(pi, s);
    pi = prof_before(PROF_LZ_C, s);
    k_blk_gs<V, B, 2><<<ntiles, RSB_BLOCK, sh, s>>>(a, t);
    RSB_CKL("k_blk_gs<2>");
    prof_after(pi, s);
  }
  (void)sh_full;
  int rc = launch_lz_eig(f32, a.units, a.S, nunits, s);
  if (rc) return rc;
  k_blk_ritz<V, B><<<ntiles, RSB_BLOCK, 0, s>>>(a);
  RSB_CKL("k_blk_ritz");
  k_blk_resid<V, B><<<ntiles, RSB_BLOCK, 0, s>>>(a);
  RSB_CKL("k_blk_resid");
  return RSB_OK;
}

static int blk_read_active(SolveBufs& SB, cudaStream_t s, int* out) {
  RSB_CK(cudaMemcpyAsync(SB.h_active, SB.n_active, sizeof(int), cudaMemcpyDeviceToHost, s));
  RSB_CK(cudaMemcpyAsync(SB.h_active + 1, &SB.gb->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  RSB_CK(cudaStreamSynchronize(s));
  prof_collect();
  *out = SB.h_active[0];
  if (SB.h_active[1] == 2)
    return rsb_set_error(RSB_ETIMEOUT,
                         "a bounded device wait gave up and a CTA's bulk copies in flight did "
                         "not drain before it exited");
  if (SB.h_active[1]) return rsb_set_error(RSB_ETIMEOUT, "a bounded device wait gave up");
  return RSB_OK;
}

// kk of a thick restart: keep + ((m - keep) mod B), so that whole blocks refill
// the basis (at most RSB_MAXKEEP)
static int blk_keep(int keep, int M, int B) {
  int kk = keep + (M - keep) % B;
  while (kk > RSB_MAXKEEP) kk -= B;
  return kk;
}

template <typename V, int B>
static int blk_run(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units, int nunits,
                   const uint64_t* ckey, SolveBufs& SB, int M, int keep, uint64_t seedbase,
                   int use_graph, cudaStream_t s) {
  BlkArgs<V> a;
  a.slice_ptr = G.slice_ptr;
  a.ent = G.ent;
  a.gid = G.gid;
  a.tiles = tiles;
  a.units = units;
  a.bu = (BlkUnit*)SB.bu;
  a.ckey = ckey;
  a.Q = (V*)SB.Q;
  a.N = SB.N;
  a.Z0 = (V*)SB.Z0;
  a.Z1 = (V*)SB.Z1;
  a.Y = (V*)SB.Y;
  a.D0 = SB.D[0];
  a.D1 = SB.D[1];
  a.partials = SB.partials;
  a.stride = ntiles;
  a.n_active = SB.n_active;
  a.stat_cycles = SB.stat_cycles;
  a.S = SB.S;
  a.seedbase = seedbase;
  a.gb = SB.gb;
  a.pb_a = prof_bytes(PROF_LZ_A);
  a.pb_a2 = prof_bytes(PROF_LZ_A2);
  a.pb_b = prof_bytes(PROF_LZ_B);
  a.pb_c = prof_bytes(PROF_LZ_C);
  const int keep_b = blk_keep(keep, M, B);
  k_blk_init<B><<<(nunits + 127) / 128, 128, 0, s>>>(units, a.bu, nunits, keep_b);
  RSB_CKL("k_blk_init");
  int active = 0;
  int rc = blk_read_active(SB, s, &active);
  if (rc || active == 0) return rc;
  RSB_CK(cudaMemsetAsync(SB.gb, 0, sizeof(GridBar), s));
  const int smax = (int)BStage<V>::bytes(M);
  RSB_CK(cudaFuncSetAttribute(k_blk_gs<V, B, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
  RSB_CK(cudaFuncSetAttribute(k_blk_gs<V, B, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
  RSB_CK(cudaFuncSetAttribute(k_blk_gs<V, B, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
  const int f32 = sizeof(V) == 4;
  cudaGraphExec_t exec = nullptr;
  std::vector<int> cap_pairs;
  if (use_graph) {
    RSB_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    prof_capture_begin();
    rc = blk_cycle<V, B>(a, ntiles, nunits, M, keep_b, f32, s);
    cap_pairs = prof_capture_end();
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return rsb_set_cuda_error(e, "cudaStreamEndCapture(block)");
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return rsb_set_cuda_error(e, "cudaGraphInstantiate(block)");
  }
  const int launches_per_cycle = 4 + 4 * (M / B) + 3;
  for (int cyc = 0; cyc < 100000; ++cyc) {
    if (exec) {
      cudaError_t e = cudaGraphLaunch(exec, s);
      rsb_count_launch(launches_per_cycle);
      if (e != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        return rsb_set_cuda_error(e, "cudaGraphLaunch(block)");
      }
      prof_replay(cap_pairs);
    } else {
      rc = blk_cycle<V, B>(a, ntiles, nunits, M, keep_b, f32, s);
      if (rc) return rc;
    }
    rc = blk_read_active(SB, s, &active);
    if (rc || active == 0) break;
  }
  if (exec) cudaGraphExecDestroy(exec);
  return rc;
}

size_t blk_unit_bytes() { return sizeof(BlkUnit); }

int solver_block_lanczos(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units,
                         int nunits, const uint64_t* ckey, SolveBufs& SB, int f32, int M, int bw,
                         int keep, uint64_t seedbase, int use_graph, cudaStream_t s) {
  if (ntiles <= 0 || nunits <= 0) return RSB_OK;
  if (!SB.Z0 || !SB.Z1 || !SB.bu) return rsb_set_error(RSB_EINVAL, "block workspace");
  const int g = use_graph ? 1 : 0;  // the block cycle runs as kernels or one CUDA graph
#define RSB_BLK_CASE(BW)                                                                         \
  case BW:                                                                                       \
    return f32 ? blk_run<float, BW>(G, tiles, ntiles, units, nunits, ckey, SB, M, keep, seedbase, \
                                    g, s)                                                        \
               : blk_run<double, BW>(G, tiles, ntiles, units, nunits, ckey, SB, M, keep,         \
                                     seedbase, g, s);
  switch (bw) {
    RSB_BLK_CASE(2)
    RSB_BLK_CASE(3)
    RSB_BLK_CASE(4)
    default:
      return rsb_set_error(RSB_EINVAL, "block width must be 1..4");
  }
#undef RSB_BLK_CASE
}
