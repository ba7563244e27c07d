// graph.cu — graph-side kernels of librsb:
//   * input validation and the CSR -> SELL-32 ingest (paper §5: the assembled
//     Laplacian; the weights are the shared-vertex counts of §2),
//   * the Laplacian action y = L x, L = D - A (paper §4),
//   * connected components of every segment (the multiplicity of the zero
//     eigenvalue, §4, decides how a half that fell apart is split),
//   * compaction: the induced subgraphs of both halves become the next level
//     (Algorithm 1: each half is bisected again),
//   * weighted cut of a candidate split (the quantity the spectral relaxation
//     of §3 minimises) and the part-id output.
#include "rsb_internal.cuh"

// ----------------------------------------------------------------------------
// validation
// ----------------------------------------------------------------------------
__global__ void k_validate(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                           const int32_t* __restrict__ wt, int64_t n, int symmetric, int* flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t b = row_ptr[i], e = row_ptr[i + 1];
  int f = 0;
  if (e < b) f |= 1;
  if (i == 0 && b != 0) f |= 1;
  for (int64_t p = b; p < e && !(f & 1); ++p) {
    const int32_t c = col[p];
    const int32_t w = wt ? wt[p] : 1;
    if (c < 0 || c >= n) { f |= 2; continue; }
    if (c == i) f |= 4;
    if (w < 1 || w > 7) f |= 8;
    if (symmetric) {
      const int64_t cb = row_ptr[c], ce = row_ptr[c + 1];
      bool found = false;
      for (int64_t q = cb; q < ce; ++q)
        if (col[q] == i && (wt ? wt[q] : 1) == w) { found = true; break; }
      if (!found) f |= 16;
    }
  }
  if (f) atomicOr(flag, f);
}

int launch_validate(const int64_t* row_ptr, const int32_t* col, const int32_t* wt, int64_t n,
                    int symmetric, int* flag, cudaStream_t s) {
  if (n <= 0) return RSB_OK;
  const int64_t nb = (n + RSB_BLOCK - 1) / RSB_BLOCK;
  k_validate<<<(unsigned)nb, RSB_BLOCK, 0, s>>>(row_ptr, col, wt, n, symmetric, flag);
  RSB_CKL("k_validate");
  return RSB_OK;
}

// ----------------------------------------------------------------------------
// SELL-32 ingest
// ----------------------------------------------------------------------------
// (perm: row i of the new order is row perm[i] of the caller's; NULL = identity)
__global__ void k_row_lengths(const int64_t* __restrict__ row_ptr, int64_t n, int32_t* len,
                              const int64_t* __restrict__ perm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t o = perm ? perm[i] : i;
  len[i] = (int32_t)(row_ptr[o + 1] - row_ptr[o]);
}

int launch_row_lengths(const int64_t* row_ptr, int64_t n, int32_t* len, cudaStream_t s,
                       const int64_t* perm) {
  if (n <= 0) return RSB_OK;
  k_row_lengths<<<(unsigned)((n + RSB_BLOCK - 1) / RSB_BLOCK), RSB_BLOCK, 0, s>>>(row_ptr, n, len,
                                                                                  perm);
  RSB_CKL("k_row_lengths");
  return RSB_OK;
}

// slice_sz[s] = 32 * (longest row of slice s); one warp per slice.
__global__ void k_slice_widths(const int32_t* __restrict__ len, int64_t n, int64_t* slice_sz) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int l = r < n ? len[r] : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l = max(l, __shfl_xor_sync(0xffffffffu, l, o));
  const int64_t nsl = (n + 31) >> 5;
  if ((threadIdx.x & 31) == 0 && (r >> 5) < nsl) slice_sz[r >> 5] = 32ll * l;
}

int launch_slice_widths(const int32_t* len, int64_t n, int64_t* slice_sz, cudaStream_t s) {
  if (n <= 0) return RSB_OK;
  const int64_t nt = ((n + 31) >> 5) << 5;
  k_slice_widths<<<(unsigned)((nt + RSB_BLOCK - 1) / RSB_BLOCK), RSB_BLOCK, 0, s>>>(len, n,
                                                                                    slice_sz);
  RSB_CKL("k_slice_widths");
  return RSB_OK;
}

__global__ void k_fill_sell(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                            const int32_t* __restrict__ wt, const int64_t* __restrict__ gid_in,
                            int64_t n, int64_t row_off, int64_t home_off, int32_t seg,
                            const int64_t* __restrict__ slice_ptr, uint32_t* __restrict__ ent,
                            int32_t* __restrict__ deg, int64_t* __restrict__ gid,
                            int64_t* __restrict__ home, int32_t* __restrict__ row_seg,
                            const int64_t* __restrict__ perm, const int32_t* __restrict__ iperm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t r = row_off + i;
  const int64_t sl = r >> 5;
  const int lane = (int)(r & 31);
  const int64_t base = slice_ptr[sl];
  const int width = (int)((slice_ptr[sl + 1] - base) >> 5);
  const int64_t o = perm ? perm[i] : i;  // the caller's row
  const int64_t b = row_ptr[o], e = row_ptr[o + 1];
  int k = 0, d = 0;
  for (int64_t p = b; p < e; ++p, ++k) {
    const uint32_t w = wt ? (uint32_t)wt[p] : 1u;
    const int64_t c = iperm ? (int64_t)iperm[col[p]] : (int64_t)col[p];
    ent[base + 32ll * k + lane] = (w << RSB_COLBITS) | (uint32_t)(c + row_off);
    d += (int)w;
  }
  for (; k < width; ++k) ent[base + 32ll * k + lane] = (uint32_t)r;  // weight 0, own column
  // the per-row arrays are optional (NULL: not wanted by the caller)
  if (deg) deg[r] = d;
  if (gid) gid[r] = gid_in ? gid_in[o] : o;
  if (home) home[r] = home_off + o;
  if (row_seg) row_seg[r] = seg;
}

int launch_fill_sell(const int64_t* row_ptr, const int32_t* col, const int32_t* wt,
                     const int64_t* gid_in, int64_t n, int64_t row_off, int64_t home_off,
                     int32_t seg, const int64_t* slice_ptr, uint32_t* ent, int32_t* deg,
                     int64_t* gid, int64_t* home, int32_t* row_seg, cudaStream_t s,
                     const int64_t* perm, const int32_t* iperm) {
  if (n <= 0) return RSB_OK;
  k_fill_sell<<<(unsigned)((n + RSB_BLOCK - 1) / RSB_BLOCK), RSB_BLOCK, 0, s>>>(
      row_ptr, col, wt, gid_in, n, row_off, home_off, seg, slice_ptr, ent, deg, gid, home,
      row_seg, perm, iperm);
  RSB_CKL("k_fill_sell");
  return RSB_OK;
}

// Padding of the last slice (rows >= n inside it) must also be harmless:
// those lanes are never read as rows, only as padding of valid rows, so
// nothing is needed there.

// ----------------------------------------------------------------------------
// exclusive scan of int64 (three-phase, recursive over block totals)
// ----------------------------------------------------------------------------
#define SCAN_ITEMS 4
#define SCAN_TILE (RSB_BLOCK * SCAN_ITEMS)

__global__ void k_scan_tiles(const int64_t* __restrict__ in, int64_t* __restrict__ out, int64_t n,
                             int64_t* __restrict__ tile_sum) {
  __shared__ int64_t sm[RSB_BLOCK];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t v[SCAN_ITEMS];
  int64_t acc = 0;
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    v[j] = (base + j < n) ? in[base + j] : 0;
    acc += v[j];
  }
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 1; o < RSB_BLOCK; o <<= 1) {
    int64_t t = threadIdx.x >= (unsigned)o ? sm[threadIdx.x - o] : 0;
    __syncthreads();
    sm[threadIdx.x] += t;
    __syncthreads();
  }
  int64_t run = sm[threadIdx.x] - acc;
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    if (base + j < n) out[base + j] = run;
    run += v[j];
  }
  if (threadIdx.x == RSB_BLOCK - 1) tile_sum[blockIdx.x] = sm[RSB_BLOCK - 1];
}

__global__ void k_scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ off) {
  const int64_t i = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x;
  const int64_t o = off[blockIdx.x];
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    const int64_t p = i + (int64_t)j * RSB_BLOCK;
    if (p < n) out[p] += o;
  }
}

size_t scan_tmp_bytes(int64_t n) {
  size_t total = 0;
  int64_t m = n;
  while (m > 1) {
    const int64_t t = (m + SCAN_TILE - 1) / SCAN_TILE;
    total += 2 * (size_t)(t + 1) * sizeof(int64_t);
    m = t;
  }
  return total + 64;
}

static int scan_rec(const int64_t* in, int64_t* out, int64_t n, int64_t* tmp, cudaStream_t s) {
  if (n <= 0) return RSB_OK;
  const int64_t t = (n + SCAN_TILE - 1) / SCAN_TILE;
  int64_t* sums = tmp;
  int64_t* offs = tmp + (t + 1);
  k_scan_tiles<<<(unsigned)t, RSB_BLOCK, 0, s>>>(in, out, n, sums);
  RSB_CKL("k_scan_tiles");
  if (t == 1) return RSB_OK;
  int rc = scan_rec(sums, offs, t, tmp + 2 * (t + 1), s);
  if (rc) return rc;
  k_scan_add<<<(unsigned)t, RSB_BLOCK, 0, s>>>(out, n, offs);
  RSB_CKL("k_scan_add");
  return RSB_OK;
}

int launch_scan_i64(const int64_t* in, int64_t* out_excl, int64_t n, void* tmp, size_t tmp_bytes,
                    cudaStream_t s) {
  if (tmp_bytes < scan_tmp_bytes(n)) return rsb_set_error(RSB_ENOMEM, "scan workspace");
  return scan_rec(in, out_excl, n, (int64_t*)tmp, s);
}

// ----------------------------------------------------------------------------
// Laplacian action on SELL-32 (building block; the solvers fuse their own)
// ----------------------------------------------------------------------------
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_spmv(const int64_t* __restrict__ slice_ptr,
                                                    const uint32_t* __restrict__ ent, int32_t n,
                                                    const V* __restrict__ x, V* __restrict__ y,
                                                    unsigned long long* pbytes) {
  const int r = blockIdx.x * RSB_BLOCK + threadIdx.x;
  int width = 0;
  if (r < n) {
    width = (int)((slice_ptr[(r >> 5) + 1] - slice_ptr[r >> 5]) >> 5);
    y[r] = spmv_row_ro<V>(slice_ptr, ent, x, r, __ldg(x + r));
  }
  if (pbytes) {  // algorithmic bytes: entries, x once, y once
    unsigned long long b = r < n ? 4ull * width + 2ull * sizeof(V) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(pbytes, b);
  }
}

int launch_spmv_f64(const LevelGraph& G, const double* x, double* y, cudaStream_t s) {
  if (G.n <= 0) return RSB_OK;
  const int pi = prof_before(PROF_SPMV, s);
  k_spmv<double><<<(G.n + RSB_BLOCK - 1) / RSB_BLOCK, RSB_BLOCK, 0, s>>>(G.slice_ptr, G.ent, G.n,
                                                                         x, y, prof_bytes(PROF_SPMV));
  RSB_CKL("k_spmv<f64>");
  prof_after(pi, s);
  return RSB_OK;
}
int launch_spmv_f32(const LevelGraph& G, const float* x, float* y, cudaStream_t s) {
  if (G.n <= 0) return RSB_OK;
  const int pi = prof_before(PROF_SPMV, s);
  k_spmv<float><<<(G.n + RSB_BLOCK - 1) / RSB_BLOCK, RSB_BLOCK, 0, s>>>(G.slice_ptr, G.ent, G.n, x,
                                                                        y, prof_bytes(PROF_SPMV));
  RSB_CKL("k_spmv<f32>");
  prof_after(pi, s);
  return RSB_OK;
}

// ----------------------------------------------------------------------------
// connected components: lock-free union-find (hook larger root under smaller)
// ----------------------------------------------------------------------------
// parent[x] <= x always holds, so every find() walk is finite; the hook retry
// loop only repeats when another thread moved a root down, which can happen
// at most x times.  Both loops carry an explicit bound anyway and raise the
// error flag if it is ever reached.
#define CC_BOUND (1 << 30)

__device__ __forceinline__ int32_t cc_find(int32_t* parent, int32_t x, int* flag) {
  int guard = 0;
  int32_t p = __ldcg(parent + x);
  while (p != x) {
    const int32_t gp = __ldcg(parent + p);
    if (gp != p) parent[x] = gp;  // path halving (benign race: gp is an ancestor)
    x = p;
    p = gp;
    if (++guard > CC_BOUND) { atomicOr(flag, 32); break; }
  }
  return x;
}

__global__ void k_cc_init(int32_t* parent, int32_t n) {
  const int r = blockIdx.x * RSB_BLOCK + threadIdx.x;
  if (r < n) parent[r] = r;
}

__global__ void k_cc_hook(const int64_t* __restrict__ slice_ptr, const uint32_t* __restrict__ ent,
                          int32_t n, int32_t* parent, int* flag) {
  const int r = blockIdx.x * RSB_BLOCK + threadIdx.x;
  if (r >= n) return;
  const int64_t base = slice_ptr[r >> 5];
  const int width = (int)((slice_ptr[(r >> 5) + 1] - base) >> 5);
  for (int k = 0; k < width; ++k) {
    const uint32_t p = ent[base + 32ll * k + (r & 31)];
    const int32_t c = (int32_t)ent_col(p);
    if (ent_w(p) == 0 || c <= r) continue;
    int32_t a = cc_find(parent, r, flag), b = cc_find(parent, c, flag);
    int guard = 0;
    while (a != b) {
      if (a < b) { const int32_t t = a; a = b; b = t; }
      const int32_t old = atomicCAS(parent + a, a, b);
      if (old == a) break;
      a = cc_find(parent, old, flag);
      b = cc_find(parent, b, flag);
      if (++guard > CC_BOUND) { atomicOr(flag, 32); break; }
    }
  }
}

__global__ void k_cc_final(int32_t* parent, int32_t n, const int64_t* __restrict__ gid,
                           unsigned long long* cmin, int* flag) {
  const int r = blockIdx.x * RSB_BLOCK + threadIdx.x;
  if (r >= n) return;
  const int32_t root = cc_find(parent, r, flag);
  atomicMin(cmin + root, (unsigned long long)gid[r]);
}

__global__ void k_cc_key(const int32_t* parent, int32_t n, const unsigned long long* cmin,
                         uint64_t* ckey, int* flag) {
  const int r = blockIdx.x * RSB_BLOCK + threadIdx.x;
  if (r >= n) return;
  const int32_t root = cc_find(const_cast<int32_t*>(parent), r, flag);
  ckey[r] = cmin[root];
}

// parent: int32[n] work; ckey: uint64[n] out (component key = smallest gid).
// `ckey` doubles as the cmin scratch (indexed by root) before the final pass;
// a second buffer is taken from the tail of `parent`'s allocation by caller.
int launch_cc(const LevelGraph& G, int32_t* parent, uint64_t* ckey, int* flag, cudaStream_t s) {
  if (G.n <= 0) return RSB_OK;
  const unsigned nb = (G.n + RSB_BLOCK - 1) / RSB_BLOCK;
  k_cc_init<<<nb, RSB_BLOCK, 0, s>>>(parent, G.n);
  RSB_CKL("k_cc_init");
  k_cc_hook<<<nb, RSB_BLOCK, 0, s>>>(G.slice_ptr, G.ent, G.n, parent, flag);
  RSB_CKL("k_cc_hook");
  RSB_CK(cudaMemsetAsync(ckey, 0xFF, sizeof(uint64_t) * (size_t)G.n, s));
  k_cc_final<<<nb, RSB_BLOCK, 0, s>>>(parent, G.n, G.gid, (unsigned long long*)ckey, flag);
  RSB_CKL("k_cc_final");
  return RSB_OK;
}

// After launch_cc, ckey[root] holds the component's smallest gid; spread it to
// every row (in place is unsafe: use a separate output).
int launch_cc_spread(const LevelGraph& G, const int32_t* parent, const uint64_t* cmin,
                     uint64_t* ckey, int* flag, cudaStream_t s) {
  if (G.n <= 0) return RSB_OK;
  const unsigned nb = (G.n + RSB_BLOCK - 1) / RSB_BLOCK;
  k_cc_key<<<nb, RSB_BLOCK, 0, s>>>(parent, G.n, (const unsigned long long*)cmin, ckey, flag);
  RSB_CKL("k_cc_key");
  return RSB_OK;
}

__global__ void k_comp_count(const int32_t* __restrict__ parent, int32_t n,
                             const int32_t* __restrict__ row_seg, int32_t* seg_ncomp) {
  const int r = blockIdx.x * RSB_BLOCK + threadIdx.x;
  if (r < n && parent[r] == r) atomicAdd(seg_ncomp + row_seg[r], 1);
}

int launch_comp_count(const LevelGraph& G, const int32_t* parent, int32_t* seg_ncomp,
                      cudaStream_t s) {
  if (G.n <= 0) return RSB_OK;
  k_comp_count<<<(G.n + RSB_BLOCK - 1) / RSB_BLOCK, RSB_BLOCK, 0, s>>>(parent, G.n, G.row_seg,
                                                                       seg_ncomp);
  RSB_CKL("k_comp_count");
  return RSB_OK;
}

// ----------------------------------------------------------------------------
// compaction into the next level (induced subgraphs of both halves)
// ----------------------------------------------------------------------------
__global__ void k_left_flag(const uint8_t* __restrict__ side, int32_t n, int64_t* flag) {
  const int r = blockIdx.x * RSB_BLOCK + threadIdx.x;
  if (r < n) flag[r] = side[r] == 0 ? 1 : 0;
}

__global__ void k_newpos(const uint8_t* __restrict__ side, int32_t n,
                         const int32_t* __restrict__ row_seg, const int64_t* __restrict__ seg_row0,
                         const int64_t* __restrict__ seg_nleft, const int64_t* __restrict__ sc,
                         int64_t* __restrict__ newpos) {
  const int r = blockIdx.x * RSB_BLOCK + threadIdx.x;
  if (r >= n) return;
  const int s = row_seg[r];
  const int64_t r0 = seg_row0[s];
  const int64_t lrank = sc[r] - sc[r0];
  newpos[r] = side[r] == 0 ? r0 + lrank : r0 + seg_nleft[s] + (r - r0 - lrank);
}

__global__ void k_newlen(const int64_t* __restrict__ slice_ptr, const uint32_t* __restrict__ ent,
                         int32_t n, const uint8_t* __restrict__ side,
                         const int64_t* __restrict__ newpos, int32_t* __restrict__ len) {
  const int r = blockIdx.x * RSB_BLOCK + threadIdx.x;
  if (r >= n) return;
  const int64_t base = slice_ptr[r >> 5];
  const int width = (int)((slice_ptr[(r >> 5) + 1] - base) >> 5);
  const uint8_t sr = side[r];
  int cnt = 0;
  for (int k = 0; k < width; ++k) {
    const uint32_t p = ent[base + 32ll * k + (r & 31)];
    if (ent_w(p) && side[ent_col(p)] == sr) ++cnt;
  }
  len[newpos[r]] = cnt;
}

__global__ void k_refill(const int64_t* __restrict__ slice_ptr, const uint32_t* __restrict__ ent,
                         const int32_t* __restrict__ deg_unused, int32_t n,
                         const uint8_t* __restrict__ side, const int64_t* __restrict__ newpos,
                         const int64_t* __restrict__ gid, const int64_t* __restrict__ home,
                         const int32_t* __restrict__ row_seg, const int32_t* __restrict__ child0,
                         const int64_t* __restrict__ nslice_ptr, uint32_t* __restrict__ nent,
                         int32_t* __restrict__ ndeg, int64_t* __restrict__ ngid,
                         int64_t* __restrict__ nhome, int32_t* __restrict__ nrow_seg) {
  const int r = blockIdx.x * RSB_BLOCK + threadIdx.x;
  if (r >= n) return;
  const int64_t base = slice_ptr[r >> 5];
  const int width = (int)((slice_ptr[(r >> 5) + 1] - base) >> 5);
  const uint8_t sr = side[r];
  const int64_t p = newpos[r];
  const int64_t nb = nslice_ptr[p >> 5];
  const int nw = (int)((nslice_ptr[(p >> 5) + 1] - nb) >> 5);
  const int lane = (int)(p & 31);
  int k2 = 0, d = 0;
  for (int k = 0; k < width; ++k) {
    const uint32_t e = ent[base + 32ll * k + (r & 31)];
    const uint32_t w = ent_w(e);
    const uint32_t c = ent_col(e);
    if (w && side[c] == sr) {
      nent[nb + 32ll * k2 + lane] = (w << RSB_COLBITS) | (uint32_t)newpos[c];
      d += (int)w;
      ++k2;
    }
  }
  for (; k2 < nw; ++k2) nent[nb + 32ll * k2 + lane] = (uint32_t)p;
  ndeg[p] = d;
  ngid[p] = gid[r];
  nhome[p] = home[r];
  nrow_seg[p] = child0[row_seg[r]] + (int32_t)sr;
}

// Builds level H from level G and the side (0 left / 1 right) of every row.
// Segment s keeps its row range; its left rows move to the front in their
// current order and its right rows follow, each row's cut edges are dropped.
// seg_child0[s] is the index of s's left child in the next level (its right
// child is seg_child0[s] + 1; an unsplit segment has only side-0 rows).
int launch_compact(const LevelGraph& G, LevelGraph& H, const uint8_t* side,
                   const int64_t* seg_row0_old, const int64_t* seg_nleft,
                   const int32_t* seg_child0, int32_t nseg, int64_t* newpos, int64_t* tmp64,
                   int32_t* len, int64_t* slice_sz, void* scan_tmp, size_t scan_tmp_bytes,
                   DevBuf& ent_buf, cudaStream_t s) {
  (void)nseg;
  const int32_t n = G.n;
  if (n <= 0) return RSB_OK;
  const unsigned nb = (n + RSB_BLOCK - 1) / RSB_BLOCK;
  k_left_flag<<<nb, RSB_BLOCK, 0, s>>>(side, n, tmp64);
  RSB_CKL("k_left_flag");
  int rc = launch_scan_i64(tmp64, tmp64, n, scan_tmp, scan_tmp_bytes, s);
  if (rc) return rc;
  k_newpos<<<nb, RSB_BLOCK, 0, s>>>(side, n, G.row_seg, seg_row0_old, seg_nleft, tmp64, newpos);
  RSB_CKL("k_newpos");
  k_newlen<<<nb, RSB_BLOCK, 0, s>>>(G.slice_ptr, G.ent, n, side, newpos, len);
  RSB_CKL("k_newlen");
  rc = launch_slice_widths(len, n, slice_sz, s);
  if (rc) return rc;
  const int64_t nsl = (n + 31) >> 5;
  RSB_CK(cudaMemsetAsync(slice_sz + nsl, 0, sizeof(int64_t), s));
  rc = launch_scan_i64(slice_sz, H.slice_ptr, nsl + 1, scan_tmp, scan_tmp_bytes, s);
  if (rc) return rc;
  int64_t total = 0;
  RSB_CK(cudaMemcpyAsync(&total, H.slice_ptr + nsl, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  RSB_CK(cudaStreamSynchronize(s));
  rc = devbuf_reserve(ent_buf, sizeof(uint32_t) * (size_t)(total > 0 ? total : 1));
  if (rc) return rc;
  H.ent = dptr<uint32_t>(ent_buf);
  H.n = n;
  H.nslices = nsl;
  H.nent = total;
  k_refill<<<nb, RSB_BLOCK, 0, s>>>(G.slice_ptr, G.ent, G.deg, n, side, newpos, G.gid, G.home,
                                    G.row_seg, seg_child0, H.slice_ptr, H.ent, H.deg, H.gid,
                                    H.home, H.row_seg);
  RSB_CKL("k_refill");
  return RSB_OK;
}

// ----------------------------------------------------------------------------
// weighted cut of candidate `cand` over each unit (sum over unit rows of the
// weights of edges whose ends got different sides, halved)
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(RSB_BLOCK)
    k_cut(const int64_t* __restrict__ slice_ptr, const uint32_t* __restrict__ ent,
          const Tile* __restrict__ tiles, Unit* units, const uint64_t* __restrict__ ckey,
          const uint8_t* __restrict__ side, int cand, double* partials, long long stride) {
  __shared__ double sm[RSB_WARPS];
  const Tile t = tiles[blockIdx.x];
  Unit& u = units[t.unit];
  if (!u.valid || cand >= u.ncand) return;
  double acc = 0.0;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    if (!unit_has(u, ckey, r)) continue;
    const int64_t base = slice_ptr[r >> 5];
    const int width = (int)((slice_ptr[(r >> 5) + 1] - base) >> 5);
    const int sr = (side[r] >> cand) & 1;
    int c = 0;
    for (int k = 0; k < width; ++k) {
      const uint32_t p = ent[base + 32ll * k + (r & 31)];
      if (((side[ent_col(p)] >> cand) & 1) != sr) c += (int)ent_w(p);
    }
    acc += (double)c;
  }
  acc = block_sum(acc, sm);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
  if (last_cta(&u.cnt, u.ntile)) {
    __shared__ double out[1];
    final_reduce(partials, stride, u.tile0, u.ntile, 1, out);
    if (threadIdx.x == 0) u.cut[cand] = (int64_t)(out[0] * 0.5);
  }
}

int launch_cut(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units,
               const uint64_t* ckey, const uint8_t* side, int cand, double* partials,
               cudaStream_t s) {
  if (ntiles <= 0) return RSB_OK;
  k_cut<<<ntiles, RSB_BLOCK, 0, s>>>(G.slice_ptr, G.ent, tiles, units, ckey, side, cand, partials,
                                     ntiles);
  RSB_CKL("k_cut");
  return RSB_OK;
}

__global__ void k_write_parts(const int64_t* __restrict__ home, const int32_t* __restrict__ row_seg,
                              int32_t n, const int32_t* __restrict__ seg_p0, int32_t* part) {
  const int r = blockIdx.x * RSB_BLOCK + threadIdx.x;
  if (r < n) part[home[r]] = seg_p0[row_seg[r]];
}

int launch_write_parts(const LevelGraph& G, const int32_t* seg_p0, int32_t* part_concat,
                       cudaStream_t s) {
  if (G.n <= 0) return RSB_OK;
  k_write_parts<<<(G.n + RSB_BLOCK - 1) / RSB_BLOCK, RSB_BLOCK, 0, s>>>(G.home, G.row_seg, G.n,
                                                                        seg_p0, part_concat);
  RSB_CKL("k_write_parts");
  return RSB_OK;
}

// ----------------------------------------------------------------------------
// recursive coordinate bisection: the coordinate of every unit row along the
// axis of the unit's largest coordinate extent (the lowest axis on equal
// extents); coords are the caller's (x, y, z) per element, indexed by home
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(RSB_BLOCK)
    k_rcb_box(const Tile* __restrict__ tiles, Unit* units, const int64_t* __restrict__ home,
              const double* __restrict__ coords, double* partials, long long stride) {
  __shared__ double sm[6][RSB_WARPS];
  __shared__ double out[6];
  const Tile t = tiles[blockIdx.x];
  Unit& u = units[t.unit];
  if (!u.valid) return;
  double m[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) m[a] = -1e300;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    const double* c = coords + 3 * home[r];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      m[a] = fmax(m[a], c[a]);
      m[3 + a] = fmax(m[3 + a], -c[a]);
    }
  }
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    const double w = warp_max(m[a]);
    if ((threadIdx.x & 31) == 0) sm[a][threadIdx.x >> 5] = w;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double b = -1e300;
    for (int i = 0; i < RSB_WARPS; ++i) b = fmax(b, sm[threadIdx.x][i]);
    partials[(long long)threadIdx.x * stride + blockIdx.x] = b;
  }
  if (last_cta(&u.cnt, u.ntile)) {
    if (threadIdx.x < 6) {
      double b = -1e300;
      for (int i = 0; i < u.ntile; ++i)
        b = fmax(b, __ldcg(partials + threadIdx.x * stride + u.tile0 + i));
      out[threadIdx.x] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int ax = 0;
      double best = out[0] + out[3];
      for (int a = 1; a < 3; ++a)
        if (out[a] + out[3 + a] > best) {
          best = out[a] + out[3 + a];
          ax = a;
        }
      u.axis = ax;
    }
  }
}

__global__ void k_rcb_vec(const Tile* __restrict__ tiles, const Unit* units,
                          const int64_t* __restrict__ home, const double* __restrict__ coords,
                          double* v) {
  const Tile t = tiles[blockIdx.x];
  const Unit& u = units[t.unit];
  if (!u.valid) return;
  const int ax = u.axis;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) v[r] = coords[3 * home[r] + ax];
}

int launch_rcb_vector(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units,
                      const double* coords, double* v, double* partials, cudaStream_t s) {
  if (ntiles <= 0) return RSB_OK;
  k_rcb_box<<<ntiles, RSB_BLOCK, 0, s>>>(tiles, units, G.home, coords, partials, ntiles);
  RSB_CKL("k_rcb_box");
  k_rcb_vec<<<ntiles, RSB_BLOCK, 0, s>>>(tiles, units, G.home, coords, v);
  RSB_CKL("k_rcb_vec");
  return RSB_OK;
}
