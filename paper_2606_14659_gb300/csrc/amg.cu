// amg.cu — the aggregation AMG V-cycle that preconditions the flexible CG of
// inverse iteration (paper §7, Algorithm 3), for all units of a level at once.
//
// Hierarchy.  Level 0 is the level's Laplacian itself (the sliced-ELL graph:
// off-diagonal -w, diagonal the weighted degree).  Level i + 1 aggregates
// pairs of consecutive rows of every unit at level i (rows 2I and 2I + 1 of
// the unit, a last odd row alone): J_i^{i+1} sums the pair, and
// L_{i+1} = J_i^{i+1} L_i J_{i+1}^i, built on the GPU in CSR (for every coarse
// row the two fine rows' entries mapped to coarse columns, sorted, duplicates
// summed: one pass counts, a scan gives row_ptr, a second pass fills).  The
// pairs follow the row order of the level, which is RCB order when the
// elements were reordered by RCB (§7 bootstraps the pairs from an RCB
// ordering).  Coarsening stops when every unit has one row; that 1 x 1
// Laplacian is 0 (its correction is 0).  Coarse values are sums of integer
// weights, exact in the vector type.
//
// V-cycle (sigma = 2/3 folded into D^-1, n_smooth = 2), at every level from the
// finest down: u = sigma D^-1 r, r -= L u, n_smooth times {du = sigma D^-1 r,
// u += du, r -= L du}; restrict r; then from the coarsest up: du = prolongated
// coarse u, u += du, r -= L du, n_smooth smoothing steps.  Level 0 runs over
// the solver's tiles (the units' rows), coarse levels over all their rows.
#include <algorithm>
#include <vector>

#include "rsb_internal.cuh"

#define AMG_SIGMA (2.0 / 3.0)
#define AMG_NSMOOTH 2
#define AMG_MAXCAND 512
#define AMG_MAXLEV 40

struct AmgLev {
  int64_t n = 0, nnz = 0;
  DevBuf rp, col, val, dinv, u, r, du;  // CSR (levels >= 1), vectors
  DevBuf cmap;                          // row -> coarse row at the next level (int32)
  DevBuf cfirst, ccnt;                  // coarse row -> first fine row, 1 or 2 (next level)
};

struct AmgWork {
  int nlev = 0;    // levels built (0: none)
  int f32 = 0;
  int64_t N = 0;   // rows of level 0
  std::vector<AmgLev> lev;
  DevBuf len, scan, flag;
};

static AmgWork g_amg[64];

static AmgWork& amg_work() {
  int dev = 0;
  cudaGetDevice(&dev);
  return g_amg[dev < 0 || dev >= 64 ? 0 : dev];
}

void amg_release() {
  for (auto& w : g_amg) {
    for (auto& l : w.lev) {
      DevBuf* all[] = {&l.rp, &l.col, &l.val, &l.dinv, &l.u, &l.r, &l.du, &l.cmap, &l.cfirst,
                       &l.ccnt};
      for (DevBuf* b : all) {
        if (b->p) cudaFree(b->p);
        b->p = nullptr;
        b->cap = 0;
      }
    }
    w.lev.clear();
    DevBuf* misc[] = {&w.len, &w.scan, &w.flag};
    for (DevBuf* b : misc) {
      if (b->p) cudaFree(b->p);
      b->p = nullptr;
      b->cap = 0;
    }
    w.nlev = 0;
  }
}

static unsigned gridn(int64_t n, int b = RSB_BLOCK) { return (unsigned)((n + b - 1) / b); }

// ----------------------------------------------------------------------------
// set-up kernels
// ----------------------------------------------------------------------------
// cmap of level 0: row r of unit u -> off1[u] + (r - row0) / 2; -1 outside units
__global__ void k_amg_map0(const Tile* __restrict__ tiles, const Unit* units,
                           const int64_t* __restrict__ off1, int32_t* cmap) {
  const Tile t = tiles[blockIdx.x];
  const Unit& u = units[t.unit];
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK)
    cmap[r] = (int32_t)(off1[t.unit] + (r - u.row0) / 2);
}

// cmap of level i >= 1 and the fine rows of every coarse row of level i + 1;
// unit u owns rows [off[u], off[u] + sz[u]) at level i.
__global__ void k_amg_map(int nunits, const int64_t* __restrict__ off,
                          const int64_t* __restrict__ sz, const int64_t* __restrict__ offc,
                          int32_t* cmap, int32_t* cfirst, int8_t* ccnt) {
  const int ui = blockIdx.y;
  if (ui >= nunits) return;
  const int64_t n = sz[ui], o = off[ui], oc = offc[ui];
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
       l += (int64_t)gridDim.x * blockDim.x) {
    cmap[o + l] = (int32_t)(oc + l / 2);
    if ((l & 1) == 0) {
      cfirst[oc + l / 2] = (int32_t)(o + l);
      ccnt[oc + l / 2] = (int8_t)(l + 1 < n ? 2 : 1);
    }
  }
}

// first fine rows of the coarse rows of level 1 (fine = level-0 rows)
__global__ void k_amg_first1(int nunits, const Unit* units, const int64_t* __restrict__ offc,
                             int32_t* cfirst, int8_t* ccnt) {
  const int ui = blockIdx.y;
  if (ui >= nunits) return;
  const Unit& u = units[ui];
  if (!u.valid) return;
  const int64_t n = u.nrows, oc = offc[ui];
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
       l += (int64_t)gridDim.x * blockDim.x)
    if ((l & 1) == 0) {
      cfirst[oc + l / 2] = (int32_t)(u.row0 + l);
      ccnt[oc + l / 2] = (int8_t)(l + 1 < n ? 2 : 1);
    }
}

// Candidates (coarse column, value) of coarse row I: the entries of its fine
// rows, columns mapped through cmap; sorted by column with equal columns
// summed.  Fine level 0 is the sliced ELL (-w off the diagonal, the degree on
// it), finer levels are CSR.  Returns the entry count or -1 on overflow.
template <typename V>
__device__ int amg_row(int64_t I, int level, const int32_t* __restrict__ cfirst,
                       const int8_t* __restrict__ ccnt, const int32_t* __restrict__ cmap,
                       const int64_t* __restrict__ slice_ptr, const uint32_t* __restrict__ ent,
                       const int32_t* __restrict__ deg, const int64_t* __restrict__ rp,
                       const int32_t* __restrict__ col, const V* __restrict__ val, int32_t* cc,
                       double* cv) {
  int nc = 0;
  const int a0 = cfirst[I];
  for (int q = 0; q < ccnt[I]; ++q) {
    const int a = a0 + q;
    if (level == 0) {
      if (nc >= AMG_MAXCAND) return -1;
      cc[nc] = cmap[a];
      cv[nc++] = (double)deg[a];
      const int64_t base = slice_ptr[a >> 5];
      const int width = (int)((slice_ptr[(a >> 5) + 1] - base) >> 5);
      for (int k = 0; k < width; ++k) {
        const uint32_t p = ent[base + 32ll * k + (a & 31)];
        if (ent_w(p) == 0) continue;
        if (nc >= AMG_MAXCAND) return -1;
        cc[nc] = cmap[ent_col(p)];
        cv[nc++] = -(double)ent_w(p);
      }
    } else {
      for (int64_t p = rp[a]; p < rp[a + 1]; ++p) {
        if (nc >= AMG_MAXCAND) return -1;
        cc[nc] = cmap[col[p]];
        cv[nc++] = (double)val[p];
      }
    }
  }
  for (int p = 1; p < nc; ++p) {  // insertion sort by column
    const int32_t x = cc[p];
    const double y = cv[p];
    int q = p - 1;
    while (q >= 0 && cc[q] > x) {
      cc[q + 1] = cc[q];
      cv[q + 1] = cv[q];
      --q;
    }
    cc[q + 1] = x;
    cv[q + 1] = y;
  }
  int m = 0;
  for (int p = 0; p < nc; ++p) {
    if (m > 0 && cc[m - 1] == cc[p]) {
      cv[m - 1] += cv[p];
    } else {
      cc[m] = cc[p];
      cv[m] = cv[p];
      ++m;
    }
  }
  return m;
}

template <typename V>
__global__ void k_amg_count(int64_t nc, int level, const int32_t* cfirst, const int8_t* ccnt,
                            const int32_t* cmap, const int64_t* slice_ptr, const uint32_t* ent,
                            const int32_t* deg, const int64_t* rp, const int32_t* col,
                            const V* val, int64_t* len, int* flag) {
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  int32_t cc[AMG_MAXCAND];
  double cv[AMG_MAXCAND];
  const int m = amg_row<V>(I, level, cfirst, ccnt, cmap, slice_ptr, ent, deg, rp, col, val, cc, cv);
  if (m < 0) {
    atomicOr(flag, 1);
    len[I] = 0;
  } else {
    len[I] = m;
  }
}

template <typename V>
__global__ void k_amg_fill(int64_t nc, int level, const int32_t* cfirst, const int8_t* ccnt,
                           const int32_t* cmap, const int64_t* slice_ptr, const uint32_t* ent,
                           const int32_t* deg, const int64_t* rp, const int32_t* col,
                           const V* val, const int64_t* rpc, int32_t* colc, V* valc, V* dinvc) {
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  int32_t cc[AMG_MAXCAND];
  double cv[AMG_MAXCAND];
  const int m = amg_row<V>(I, level, cfirst, ccnt, cmap, slice_ptr, ent, deg, rp, col, val, cc, cv);
  if (m < 0) return;
  int64_t o = rpc[I];
  double d = 0.0;
  for (int p = 0; p < m; ++p) {
    colc[o + p] = cc[p];
    valc[o + p] = V(cv[p]);
    if (cc[p] == (int32_t)I) d = cv[p];
  }
  dinvc[I] = d > 0.0 ? V(AMG_SIGMA / d) : V(0);
}

// ----------------------------------------------------------------------------
// V-cycle kernels
// ----------------------------------------------------------------------------
// level 0 (tiles over the units' rows; D from the weighted degree)
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_vc0_start(const Tile* __restrict__ tiles,
                                                       const Unit* units,
                                                       const int32_t* __restrict__ deg,
                                                       const V* __restrict__ rin, V* r, V* u,
                                                       V* du) {
  const Tile t = tiles[blockIdx.x];
  if (units[t.unit].status != U_ACTIVE) return;
  for (int i = t.row0 + threadIdx.x; i < t.row1; i += RSB_BLOCK) {
    const V ri = rin[i];
    const V d = deg[i] > 0 ? V(AMG_SIGMA / (double)deg[i]) : V(0);
    r[i] = ri;
    u[i] = d * ri;
    du[i] = d * ri;
  }
}

template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_vc0_resid(const Tile* __restrict__ tiles,
                                                       const Unit* units,
                                                       const int64_t* __restrict__ slice_ptr,
                                                       const uint32_t* __restrict__ ent,
                                                       const V* __restrict__ du, V* r) {
  const Tile t = tiles[blockIdx.x];
  if (units[t.unit].status != U_ACTIVE) return;
  for (int i = t.row0 + threadIdx.x; i < t.row1; i += RSB_BLOCK)
    r[i] -= spmv_row_ro<V>(slice_ptr, ent, du, i, du[i]);
}

// mode 0: du = sigma D^-1 r, u += du; mode 1: du = coarse u at the row's
// aggregate, u += du
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_vc0_step(const Tile* __restrict__ tiles,
                                                      const Unit* units,
                                                      const int32_t* __restrict__ deg,
                                                      const int32_t* __restrict__ cmap,
                                                      const V* __restrict__ uc, int mode,
                                                      const V* __restrict__ r, V* u, V* du) {
  const Tile t = tiles[blockIdx.x];
  if (units[t.unit].status != U_ACTIVE) return;
  for (int i = t.row0 + threadIdx.x; i < t.row1; i += RSB_BLOCK) {
    V d;
    if (mode == 0) d = deg[i] > 0 ? V(AMG_SIGMA / (double)deg[i]) * r[i] : V(0);
    else d = uc[cmap[i]];
    du[i] = d;
    u[i] += d;
  }
}

// coarse levels (CSR, all rows)
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_vc_start(int64_t n, const V* __restrict__ dinv,
                                                      V* r, V* u, V* du) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const V d = dinv[i] * r[i];
  u[i] = d;
  du[i] = d;
}

template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_vc_resid(int64_t n, const int64_t* __restrict__ rp,
                                                      const int32_t* __restrict__ col,
                                                      const V* __restrict__ val,
                                                      const V* __restrict__ du, V* r) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  V acc = V(0);
  for (int64_t p = rp[i]; p < rp[i + 1]; ++p) acc += val[p] * __ldg(du + col[p]);
  r[i] -= acc;
}

template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_vc_step(int64_t n, const V* __restrict__ dinv,
                                                     const int32_t* __restrict__ cmap,
                                                     const V* __restrict__ uc, int mode,
                                                     const V* __restrict__ r, V* u, V* du) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const V d = mode == 0 ? dinv[i] * r[i] : uc[cmap[i]];
  du[i] = d;
  u[i] += d;
}

// r_c[I] = sum of r over the fine rows of coarse row I
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_vc_restrict(int64_t nc, const int32_t* __restrict__ cfirst,
                                                         const int8_t* __restrict__ ccnt,
                                                         const V* __restrict__ rf, V* rc) {
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  const int a = cfirst[I];
  rc[I] = ccnt[I] == 2 ? rf[a] + rf[a + 1] : rf[a];
}

// ----------------------------------------------------------------------------
// host: set-up and application
// ----------------------------------------------------------------------------
template <typename V>
static int amg_setup_t(const LevelGraph& G, const Tile* tiles, int ntiles, const Unit* units,
                       const std::vector<Unit>& hunits, cudaStream_t s) {
  AmgWork& w = amg_work();
  w.nlev = 0;
  w.f32 = sizeof(V) == 4;
  w.N = G.n;
  const int nunits = (int)hunits.size();
  if (w.lev.size() < AMG_MAXLEV) w.lev.resize(AMG_MAXLEV);
  // per-unit sizes of every level
  std::vector<std::vector<int64_t>> sz(1), off(1);
  for (const Unit& u : hunits) sz[0].push_back(u.valid ? u.nrows : 0);
  int rc;
  DevBuf dev_off, dev_sz;  // per level, uploaded on demand
  AmgLev& L0 = w.lev[0];
  L0.n = G.n;
  const size_t es = sizeof(V);
  if ((rc = devbuf_reserve(L0.u, es * (size_t)(G.n + 32))) ||
      (rc = devbuf_reserve(L0.r, es * (size_t)(G.n + 32))) ||
      (rc = devbuf_reserve(L0.du, es * (size_t)(G.n + 32))) ||
      (rc = devbuf_reserve(L0.cmap, sizeof(int32_t) * (size_t)(G.n + 32))) ||
      (rc = devbuf_reserve(w.flag, 64)))
    return rc;
  int nlev = 1;
  for (int i = 0; i + 1 < AMG_MAXLEV; ++i) {
    // next level's sizes and offsets
    std::vector<int64_t> szc(nunits), offc(nunits);
    int64_t nc = 0, maxsz = 0;
    for (int ui = 0; ui < nunits; ++ui) {
      maxsz = std::max(maxsz, sz[i][ui]);
      szc[ui] = (sz[i][ui] + 1) / 2;
      offc[ui] = nc;
      nc += szc[ui];
    }
    if (maxsz <= 1) break;  // every unit is down to one row
    std::vector<int64_t> offi(nunits);
    {
      int64_t o = 0;
      for (int ui = 0; ui < nunits; ++ui) {
        offi[ui] = o;
        o += sz[i][ui];
      }
    }
    AmgLev& F = w.lev[i];
    AmgLev& C = w.lev[i + 1];
    C.n = nc;
    if ((rc = devbuf_reserve(F.cfirst, sizeof(int32_t) * (size_t)(nc + 1))) ||
        (rc = devbuf_reserve(F.ccnt, (size_t)(nc + 1))) ||
        (rc = devbuf_reserve(C.rp, sizeof(int64_t) * (size_t)(nc + 2))) ||
        (rc = devbuf_reserve(C.dinv, es * (size_t)(nc + 1))) ||
        (rc = devbuf_reserve(C.u, es * (size_t)(nc + 1))) ||
        (rc = devbuf_reserve(C.r, es * (size_t)(nc + 1))) ||
        (rc = devbuf_reserve(C.du, es * (size_t)(nc + 1))) ||
        (rc = devbuf_reserve(C.cmap, sizeof(int32_t) * (size_t)(nc + 1))) ||
        (rc = devbuf_reserve(w.len, sizeof(int64_t) * (size_t)(nc + 2))) ||
        (rc = devbuf_reserve(w.scan, scan_tmp_bytes(nc + 2))) ||
        (rc = devbuf_reserve(dev_off, sizeof(int64_t) * 3 * (size_t)nunits)))
      return rc;
    int64_t* d_offi = dptr<int64_t>(dev_off);
    int64_t* d_szi = d_offi + nunits;
    int64_t* d_offc = d_szi + nunits;
    RSB_CK(cudaMemcpyAsync(d_offi, offi.data(), sizeof(int64_t) * nunits, cudaMemcpyHostToDevice, s));
    RSB_CK(cudaMemcpyAsync(d_szi, sz[i].data(), sizeof(int64_t) * nunits, cudaMemcpyHostToDevice, s));
    RSB_CK(cudaMemcpyAsync(d_offc, offc.data(), sizeof(int64_t) * nunits, cudaMemcpyHostToDevice, s));
    const dim3 gmap((unsigned)std::min<int64_t>(1024, std::max<int64_t>(1, (maxsz + 255) / 256)),
                    (unsigned)nunits);
    if (i == 0) {
      k_amg_map0<<<ntiles, RSB_BLOCK, 0, s>>>(tiles, units, d_offc, dptr<int32_t>(F.cmap));
      RSB_CKL("k_amg_map0");
      k_amg_first1<<<gmap, RSB_BLOCK, 0, s>>>(nunits, units, d_offc, dptr<int32_t>(F.cfirst),
                                              dptr<int8_t>(F.ccnt));
      RSB_CKL("k_amg_first1");
    } else {
      k_amg_map<<<gmap, RSB_BLOCK, 0, s>>>(nunits, d_offi, d_szi, d_offc, dptr<int32_t>(F.cmap),
                                           dptr<int32_t>(F.cfirst), dptr<int8_t>(F.ccnt));
      RSB_CKL("k_amg_map");
    }
    RSB_CK(cudaMemsetAsync(w.flag.p, 0, sizeof(int), s));
    int64_t* len = dptr<int64_t>(w.len);
    k_amg_count<V><<<gridn(nc, 128), 128, 0, s>>>(
        nc, i, dptr<int32_t>(F.cfirst), dptr<int8_t>(F.ccnt), dptr<int32_t>(F.cmap), G.slice_ptr,
        G.ent, G.deg, i ? dptr<int64_t>(F.rp) : nullptr, i ? dptr<int32_t>(F.col) : nullptr,
        i ? dptr<V>(F.val) : nullptr, len, dptr<int>(w.flag));
    RSB_CKL("k_amg_count");
    RSB_CK(cudaMemsetAsync(len + nc, 0, sizeof(int64_t), s));
    if ((rc = launch_scan_i64(len, dptr<int64_t>(C.rp), nc + 1, w.scan.p, w.scan.cap, s))) return rc;
    int64_t nnz = 0;
    int flag = 0;
    RSB_CK(cudaMemcpyAsync(&nnz, dptr<int64_t>(C.rp) + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    RSB_CK(cudaMemcpyAsync(&flag, w.flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    RSB_CK(cudaStreamSynchronize(s));
    if (flag) break;  // a coarse row too wide to build: level i is the coarsest (correction 0)
    C.nnz = nnz;
    if ((rc = devbuf_reserve(C.col, sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1))) ||
        (rc = devbuf_reserve(C.val, es * (size_t)std::max<int64_t>(nnz, 1))))
      return rc;
    k_amg_fill<V><<<gridn(nc, 128), 128, 0, s>>>(
        nc, i, dptr<int32_t>(F.cfirst), dptr<int8_t>(F.ccnt), dptr<int32_t>(F.cmap), G.slice_ptr,
        G.ent, G.deg, i ? dptr<int64_t>(F.rp) : nullptr, i ? dptr<int32_t>(F.col) : nullptr,
        i ? dptr<V>(F.val) : nullptr, dptr<int64_t>(C.rp), dptr<int32_t>(C.col), dptr<V>(C.val),
        dptr<V>(C.dinv));
    RSB_CKL("k_amg_fill");
    sz.push_back(szc);
    off.push_back(offc);
    nlev = i + 2;
  }
  RSB_CK(cudaStreamSynchronize(s));
  if (dev_off.p) cudaFree(dev_off.p);
  w.nlev = nlev;
  return RSB_OK;
}

// z = V-cycle(r) on the units' rows of level 0 (both level-0 vectors N long)
template <typename V>
static int amg_apply_t(const LevelGraph& G, const Tile* tiles, int ntiles, const Unit* units,
                       const V* rin, V* z, cudaStream_t s) {
  AmgWork& w = amg_work();
  const int K = w.nlev;
  AmgLev& L0 = w.lev[0];
  V* u0 = z;
  V* r0 = dptr<V>(L0.r);
  V* du0 = dptr<V>(L0.du);
  // descend
  for (int i = 0; i < K; ++i) {
    AmgLev& Li = w.lev[i];
    const bool last = i + 1 == K;
    if (i == 0) {
      k_vc0_start<V><<<ntiles, RSB_BLOCK, 0, s>>>(tiles, units, G.deg, rin, r0, u0, du0);
      RSB_CKL("k_vc0_start");
      k_vc0_resid<V><<<ntiles, RSB_BLOCK, 0, s>>>(tiles, units, G.slice_ptr, G.ent, du0, r0);
      RSB_CKL("k_vc0_resid");
      for (int sm = 0; sm < AMG_NSMOOTH; ++sm) {
        k_vc0_step<V><<<ntiles, RSB_BLOCK, 0, s>>>(tiles, units, G.deg, nullptr, nullptr, 0, r0,
                                                   u0, du0);
        RSB_CKL("k_vc0_step");
        k_vc0_resid<V><<<ntiles, RSB_BLOCK, 0, s>>>(tiles, units, G.slice_ptr, G.ent, du0, r0);
        RSB_CKL("k_vc0_resid");
      }
    } else {
      const int64_t n = Li.n;
      V* r = dptr<V>(Li.r);
      V* u = dptr<V>(Li.u);
      V* du = dptr<V>(Li.du);
      k_vc_start<V><<<gridn(n), RSB_BLOCK, 0, s>>>(n, dptr<V>(Li.dinv), r, u, du);
      RSB_CKL("k_vc_start");
      if (last) continue;  // the coarsest level: one Jacobi step (a 1 x 1 zero gives 0)
      k_vc_resid<V><<<gridn(n), RSB_BLOCK, 0, s>>>(n, dptr<int64_t>(Li.rp), dptr<int32_t>(Li.col),
                                                   dptr<V>(Li.val), du, r);
      RSB_CKL("k_vc_resid");
      for (int sm = 0; sm < AMG_NSMOOTH; ++sm) {
        k_vc_step<V><<<gridn(n), RSB_BLOCK, 0, s>>>(n, dptr<V>(Li.dinv), nullptr, nullptr, 0, r,
                                                    u, du);
        RSB_CKL("k_vc_step");
        k_vc_resid<V><<<gridn(n), RSB_BLOCK, 0, s>>>(n, dptr<int64_t>(Li.rp),
                                                     dptr<int32_t>(Li.col), dptr<V>(Li.val), du, r);
        RSB_CKL("k_vc_resid");
      }
    }
    if (!last) {
      AmgLev& C = w.lev[i + 1];
      k_vc_restrict<V><<<gridn(C.n), RSB_BLOCK, 0, s>>>(C.n, dptr<int32_t>(Li.cfirst),
                                                        dptr<int8_t>(Li.ccnt),
                                                        i == 0 ? r0 : dptr<V>(Li.r), dptr<V>(C.r));
      RSB_CKL("k_vc_restrict");
    }
  }
  // ascend
  for (int i = K - 2; i >= 0; --i) {
    AmgLev& Li = w.lev[i];
    AmgLev& C = w.lev[i + 1];
    if (i == 0) {
      k_vc0_step<V><<<ntiles, RSB_BLOCK, 0, s>>>(tiles, units, G.deg, dptr<int32_t>(L0.cmap),
                                                 dptr<V>(C.u), 1, r0, u0, du0);
      RSB_CKL("k_vc0_step(prolong)");
      k_vc0_resid<V><<<ntiles, RSB_BLOCK, 0, s>>>(tiles, units, G.slice_ptr, G.ent, du0, r0);
      RSB_CKL("k_vc0_resid");
      for (int sm = 0; sm < AMG_NSMOOTH; ++sm) {
        k_vc0_step<V><<<ntiles, RSB_BLOCK, 0, s>>>(tiles, units, G.deg, nullptr, nullptr, 0, r0,
                                                   u0, du0);
        RSB_CKL("k_vc0_step");
        if (sm + 1 < AMG_NSMOOTH) {
          k_vc0_resid<V><<<ntiles, RSB_BLOCK, 0, s>>>(tiles, units, G.slice_ptr, G.ent, du0, r0);
          RSB_CKL("k_vc0_resid");
        }
      }
    } else {
      const int64_t n = Li.n;
      V* r = dptr<V>(Li.r);
      V* u = dptr<V>(Li.u);
      V* du = dptr<V>(Li.du);
      k_vc_step<V><<<gridn(n), RSB_BLOCK, 0, s>>>(n, dptr<V>(Li.dinv), dptr<int32_t>(Li.cmap),
                                                  dptr<V>(C.u), 1, r, u, du);
      RSB_CKL("k_vc_step(prolong)");
      k_vc_resid<V><<<gridn(n), RSB_BLOCK, 0, s>>>(n, dptr<int64_t>(Li.rp), dptr<int32_t>(Li.col),
                                                   dptr<V>(Li.val), du, r);
      RSB_CKL("k_vc_resid");
      for (int sm = 0; sm < AMG_NSMOOTH; ++sm) {
        k_vc_step<V><<<gridn(n), RSB_BLOCK, 0, s>>>(n, dptr<V>(Li.dinv), nullptr, nullptr, 0, r,
                                                    u, du);
        RSB_CKL("k_vc_step");
        k_vc_resid<V><<<gridn(n), RSB_BLOCK, 0, s>>>(n, dptr<int64_t>(Li.rp),
                                                     dptr<int32_t>(Li.col), dptr<V>(Li.val), du, r);
        RSB_CKL("k_vc_resid");
      }
    }
  }
  return RSB_OK;
}

int amg_setup(int f32, const LevelGraph& G, const Tile* tiles, int ntiles, const Unit* units,
              const std::vector<Unit>& hunits, cudaStream_t s) {
  return f32 ? amg_setup_t<float>(G, tiles, ntiles, units, hunits, s)
             : amg_setup_t<double>(G, tiles, ntiles, units, hunits, s);
}

int amg_levels() { return amg_work().nlev; }

int amg_apply(int f32, const LevelGraph& G, const Tile* tiles, int ntiles, const Unit* units,
              const void* r, void* z, cudaStream_t s) {
  if (amg_work().nlev < 1) return rsb_set_error(RSB_EINVAL, "AMG hierarchy not set up");
  return f32 ? amg_apply_t<float>(G, tiles, ntiles, units, (const float*)r, (float*)z, s)
             : amg_apply_t<double>(G, tiles, ntiles, units, (const double*)r, (double*)z, s);
}
