// select.cu — the median split of Algorithm 1 (§4), done as a selection
// instead of the sort the paper describes:
//   * orientation of the Fiedler vector (reading R4: the smallest gid among
//     |v| >= max|v|/2 must come out negative),
//   * a segmented 8-bit-digit radix select of the k-th smallest key per unit
//     (keys: order-preserving bits of the FP64 value, a gid, or a component
//     key), which gives the same answer as sorting and taking k elements,
//   * the tie window of reading R7 (values within tie_rel * range of the k-th
//     value are ties and go left in ascending gid),
//   * the gid rule comparing two candidate splits of a repeated eigenvalue
//     (reading R5), and the final side of every row including whole
//     components placed by reading R8.
#include "rsb_internal.cuh"

// ----------------------------------------------------------------------------
// per-unit max weighted degree (the ||L|| scale of the stopping tests)
// ----------------------------------------------------------------------------
__device__ __forceinline__ void final_max(const double* partials, long long stride, int t0, int nt,
                                          double* out) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w == 0) {
    double m = -1e300;
    for (int t = lane; t < nt; t += 32) m = fmax(m, __ldcg(partials + stride * 0 + t0 + t));
    m = warp_max(m);
    if (lane == 0) out[0] = m;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(RSB_BLOCK)
    k_degree_max(const int32_t* __restrict__ deg, const Tile* __restrict__ tiles, Unit* units,
                 const uint64_t* __restrict__ ckey, double* partials, long long stride) {
  __shared__ double sm[RSB_WARPS];
  __shared__ double out[1];
  const Tile t = tiles[blockIdx.x];
  Unit& u = units[t.unit];
  if (!u.valid) return;
  double m = 0.0;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK)
    if (unit_has(u, ckey, r)) m = fmax(m, (double)deg[r]);
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int i = 0; i < RSB_WARPS; ++i) b = fmax(b, sm[i]);
    partials[blockIdx.x] = b;
  }
  if (last_cta(&u.cnt, u.ntile)) {
    final_max(partials, stride, u.tile0, u.ntile, out);
    if (threadIdx.x == 0) u.dmax = out[0];
  }
}

int launch_degree_max(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units,
                      const uint64_t* ckey, double* partials, cudaStream_t s) {
  if (ntiles <= 0) return RSB_OK;
  k_degree_max<<<ntiles, RSB_BLOCK, 0, s>>>(G.deg, tiles, units, ckey, partials, ntiles);
  RSB_CKL("k_degree_max");
  return RSB_OK;
}

// ----------------------------------------------------------------------------
// orientation statistics: amax = max|v|, vmax, vmin over the unit
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(RSB_BLOCK)
    k_orient_stats(const Tile* __restrict__ tiles, Unit* units, const uint64_t* __restrict__ ckey,
                   const double* __restrict__ v, int cand, double* partials, long long stride) {
  __shared__ double sm[3][RSB_WARPS];
  __shared__ double out[3];
  const Tile t = tiles[blockIdx.x];
  Unit& u = units[t.unit];
  if (!u.valid || cand >= u.ncand) return;
  double a = 0.0, hi = -1e300, lo = 1e300;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    if (!unit_has(u, ckey, r)) continue;
    const double x = v[r];
    a = fmax(a, fabs(x));
    hi = fmax(hi, x);
    lo = fmin(lo, x);
  }
  a = warp_max(a);
  hi = warp_max(hi);
  lo = -warp_max(-lo);
  if ((threadIdx.x & 31) == 0) {
    sm[0][threadIdx.x >> 5] = a;
    sm[1][threadIdx.x >> 5] = hi;
    sm[2][threadIdx.x >> 5] = -lo;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double b = -1e300;
    for (int i = 0; i < RSB_WARPS; ++i) b = fmax(b, sm[threadIdx.x][i]);
    partials[(long long)threadIdx.x * stride + blockIdx.x] = b;
  }
  if (last_cta(&u.cnt, u.ntile)) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w < 3) {
      double m = -1e300;
      for (int i = lane; i < u.ntile; i += 32) m = fmax(m, __ldcg(partials + w * stride + u.tile0 + i));
      m = warp_max(m);
      if (lane == 0) out[w] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      u.amax = out[0];
      u.vmax = out[1];
      u.vmin = -out[2];
    }
  }
}

// g* = smallest gid among rows with |v| >= amax / 2, and v at g*; then the
// sign that makes v[g*] negative and the tie window tau.
__global__ void __launch_bounds__(RSB_BLOCK)
    k_orient_gstar(const int64_t* __restrict__ gid, const Tile* __restrict__ tiles, Unit* units,
                   const uint64_t* __restrict__ ckey, const double* __restrict__ v, int cand,
                   double tie_rel, double* partials, long long stride, int fixed_sign) {
  __shared__ long long smg[RSB_WARPS];
  __shared__ double smv[RSB_WARPS];
  const Tile t = tiles[blockIdx.x];
  Unit& u = units[t.unit];
  if (!u.valid || cand >= u.ncand) return;
  const double thr = 0.5 * u.amax;
  long long g = LLONG_MAX;
  double gv = 0.0;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    if (!unit_has(u, ckey, r)) continue;
    const double x = v[r];
    if (fabs(x) >= thr && gid[r] < g) {
      g = gid[r];
      gv = x;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long og = __shfl_xor_sync(0xffffffffu, g, o);
    const double ov = __shfl_xor_sync(0xffffffffu, gv, o);
    if (og < g) { g = og; gv = ov; }
  }
  if ((threadIdx.x & 31) == 0) {
    smg[threadIdx.x >> 5] = g;
    smv[threadIdx.x >> 5] = gv;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < RSB_WARPS; ++i)
      if (smg[i] < g) { g = smg[i]; gv = smv[i]; }
    partials[blockIdx.x] = (double)g;
    partials[stride + blockIdx.x] = gv;
  }
  if (last_cta(&u.cnt, u.ntile)) {
    if (threadIdx.x == 0) {
      double bg = 1e300, bv = 0.0;
      for (int i = 0; i < u.ntile; ++i) {
        const double pg = __ldcg(partials + u.tile0 + i);
        if (pg < bg) { bg = pg; bv = __ldcg(partials + stride + u.tile0 + i); }
      }
      u.gstar = (int64_t)bg;
      u.gstar_v = bv;
      u.sign = fixed_sign ? 1.0 : (bv > 0.0 ? -1.0 : 1.0);
      u.tau = tie_rel * (u.vmax - u.vmin);
    }
  }
}

// fixed_sign: keep v as it is (RCB: lower coordinates go left)
int launch_orient(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units,
                  const uint64_t* ckey, const double* v, int cand, double tie_rel,
                  double* partials, cudaStream_t s, int fixed_sign) {
  if (ntiles <= 0) return RSB_OK;
  k_orient_stats<<<ntiles, RSB_BLOCK, 0, s>>>(tiles, units, ckey, v, cand, partials, ntiles);
  RSB_CKL("k_orient_stats");
  k_orient_gstar<<<ntiles, RSB_BLOCK, 0, s>>>(G.gid, tiles, units, ckey, v, cand, tie_rel,
                                              partials, ntiles, fixed_sign);
  RSB_CKL("k_orient_gstar");
  return RSB_OK;
}

// ----------------------------------------------------------------------------
// segmented radix select
// ----------------------------------------------------------------------------
// mode 0: key = order bits of sign * v over unit rows, rank u.k        -> u.vk
// mode 1: key = gid over tie rows (|sign v - vk| <= tau), rank k-below -> u.sel_prefix
// mode 2: key = component key over all unit rows, rank u.k           -> u.sel_prefix
enum { SEL_VALUE = 0, SEL_TIEGID = 1, SEL_COMP = 2 };

__device__ __forceinline__ bool sel_member(const Unit& u, int mode, int r, const uint64_t* ckey,
                                           const double* v, const int64_t* gid, uint64_t& key) {
  if (mode == SEL_COMP) {
    key = ckey[r];
    return true;
  }
  if (!unit_has(u, ckey, r)) return false;
  const double x = u.sign * v[r];
  if (mode == SEL_VALUE) {
    key = dkey(x);
    return true;
  }
  if (fabs(x - u.vk) <= u.tau) {
    key = (uint64_t)gid[r];
    return true;
  }
  return false;
}

__global__ void k_sel_init(Unit* units, int nunits, int mode, int cand) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nunits) return;
  Unit& u = units[i];
  if (!u.valid || (mode != SEL_COMP && cand >= u.ncand)) return;
  u.sel_prefix = 0;
  u.sel_below = 0;
  u.sel_eq = 0;
  u.sel_k = (mode == SEL_TIEGID) ? (u.k - u.below) : u.k;
}

__global__ void __launch_bounds__(RSB_BLOCK)
    k_sel_hist(const int64_t* __restrict__ gid, const Tile* __restrict__ tiles, const Unit* units,
               const uint64_t* __restrict__ ckey, const double* __restrict__ v, int mode, int cand,
               int shift, int* __restrict__ hist) {
  __shared__ int sh[256];
  const Tile t = tiles[blockIdx.x];
  const Unit& u = units[t.unit];
  if (!u.valid || (mode != SEL_COMP && cand >= u.ncand)) return;
  sh[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t himask = shift >= 56 ? 0ull : (~0ull << (shift + 8));
  const uint64_t want = u.sel_prefix & himask;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    uint64_t key;
    if (!sel_member(u, mode, r, ckey, v, gid, key)) continue;
    if ((key & himask) != want) continue;
    atomicAdd(&sh[(key >> shift) & 255u], 1);
  }
  __syncthreads();
  const int c = sh[threadIdx.x];
  if (c) atomicAdd(hist + (long long)t.unit * 256 + threadIdx.x, c);
}

__global__ void __launch_bounds__(256) k_sel_scan(Unit* units, int mode, int cand, int shift,
                                                  int* hist) {
  __shared__ int sc[256];
  Unit& u = units[blockIdx.x];
  if (!u.valid || (mode != SEL_COMP && cand >= u.ncand)) return;
  int* h = hist + (long long)blockIdx.x * 256;
  const int c = h[threadIdx.x];
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    const int x = threadIdx.x >= (unsigned)o ? sc[threadIdx.x - o] : 0;
    __syncthreads();
    sc[threadIdx.x] += x;
    __syncthreads();
  }
  const long long incl = sc[threadIdx.x];
  const long long excl = incl - c;
  const long long k = u.sel_k;
  if (c > 0 && excl < k && k <= incl) {
    u.sel_k = k - excl;
    u.sel_below += excl;
    u.sel_prefix |= (uint64_t)threadIdx.x << shift;
    u.sel_eq = c;
    if (shift == 0 && mode == SEL_VALUE) u.vk = dkey_inv(u.sel_prefix);
  }
  h[threadIdx.x] = 0;
}

int launch_select(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units, int nunits,
                  const uint64_t* ckey, const double* v, int mode, int cand, int* hist,
                  cudaStream_t s) {
  if (ntiles <= 0 || nunits <= 0) return RSB_OK;
  k_sel_init<<<(nunits + 255) / 256, 256, 0, s>>>(units, nunits, mode, cand);
  RSB_CKL("k_sel_init");
  for (int shift = 56; shift >= 0; shift -= 8) {
    k_sel_hist<<<ntiles, RSB_BLOCK, 0, s>>>(G.gid, tiles, units, ckey, v, mode, cand, shift, hist);
    RSB_CKL("k_sel_hist");
    k_sel_scan<<<nunits, 256, 0, s>>>(units, mode, cand, shift, hist);
    RSB_CKL("k_sel_scan");
  }
  return RSB_OK;
}

// ----------------------------------------------------------------------------
// R7: rows strictly below the tie window, then the side bit of candidate cand
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(RSB_BLOCK)
    k_split_below(const Tile* __restrict__ tiles, Unit* units, const uint64_t* __restrict__ ckey,
                  const double* __restrict__ v, int cand, double* partials, long long stride) {
  __shared__ double sm[RSB_WARPS];
  __shared__ double out[1];
  const Tile t = tiles[blockIdx.x];
  Unit& u = units[t.unit];
  if (!u.valid || cand >= u.ncand) return;
  const double lim = u.vk - u.tau;
  double c = 0.0;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK)
    if (unit_has(u, ckey, r) && u.sign * v[r] < lim) c += 1.0;
  c = block_sum(c, sm);
  if (threadIdx.x == 0) partials[blockIdx.x] = c;
  if (last_cta(&u.cnt, u.ntile)) {
    final_reduce(partials, stride, u.tile0, u.ntile, 1, out);
    if (threadIdx.x == 0) u.below = (int64_t)out[0];
  }
}

int launch_split_below(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units,
                       const uint64_t* ckey, const double* v, int cand, double* partials,
                       cudaStream_t s) {
  (void)G;
  if (ntiles <= 0) return RSB_OK;
  k_split_below<<<ntiles, RSB_BLOCK, 0, s>>>(tiles, units, ckey, v, cand, partials, ntiles);
  RSB_CKL("k_split_below");
  return RSB_OK;
}

__global__ void __launch_bounds__(RSB_BLOCK)
    k_split_assign(const int64_t* __restrict__ gid, const Tile* __restrict__ tiles,
                   const Unit* units, const uint64_t* __restrict__ ckey,
                   const double* __restrict__ v, int cand, uint8_t* side) {
  const Tile t = tiles[blockIdx.x];
  const Unit& u = units[t.unit];
  if (!u.valid || cand >= u.ncand) return;
  const double lim = u.vk - u.tau;
  const uint64_t gthr = u.sel_prefix;  // k''-th smallest tie gid
  const bool all_below = (u.k - u.below) <= 0;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    if (!unit_has(u, ckey, r)) continue;
    const double x = u.sign * v[r];
    bool left = x < lim;
    if (!left && !all_below && fabs(x - u.vk) <= u.tau) left = (uint64_t)gid[r] <= gthr;
    const uint8_t bit = (uint8_t)(1u << cand);
    side[r] = left ? (uint8_t)(side[r] & ~bit) : (uint8_t)(side[r] | bit);
  }
}

int launch_split_assign(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units,
                        const uint64_t* ckey, const double* v, uint8_t* side, int cand,
                        cudaStream_t s) {
  if (ntiles <= 0) return RSB_OK;
  k_split_assign<<<ntiles, RSB_BLOCK, 0, s>>>(G.gid, tiles, units, ckey, v, cand, side);
  RSB_CKL("k_split_assign");
  return RSB_OK;
}

// ----------------------------------------------------------------------------
// R5 gid rule: smallest gid where candidates a and b disagree, and whether a
// has it on the left.  Result: u.best updated (a wins -> a, else b) among
// candidates of equal cut; the caller runs it after comparing cuts.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(RSB_BLOCK)
    k_choose(const int64_t* __restrict__ gid, const Tile* __restrict__ tiles, Unit* units,
             const uint64_t* __restrict__ ckey, const uint8_t* __restrict__ side, int cb,
             double* partials, long long stride) {
  __shared__ long long smg[RSB_WARPS];
  __shared__ int sml[RSB_WARPS];
  const Tile t = tiles[blockIdx.x];
  Unit& u = units[t.unit];
  if (!u.valid || cb >= u.ncand) return;
  const int ca = u.best;
  long long g = LLONG_MAX;
  int aleft = 0;
  for (int r = t.row0 + threadIdx.x; r < t.row1; r += RSB_BLOCK) {
    if (!unit_has(u, ckey, r)) continue;
    const int sa = (side[r] >> ca) & 1, sb = (side[r] >> cb) & 1;
    if (sa != sb && gid[r] < g) {
      g = gid[r];
      aleft = sa == 0;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long og = __shfl_xor_sync(0xffffffffu, g, o);
    const int ol = __shfl_xor_sync(0xffffffffu, aleft, o);
    if (og < g) { g = og; aleft = ol; }
  }
  if ((threadIdx.x & 31) == 0) {
    smg[threadIdx.x >> 5] = g;
    sml[threadIdx.x >> 5] = aleft;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < RSB_WARPS; ++i)
      if (smg[i] < g) { g = smg[i]; aleft = sml[i]; }
    partials[blockIdx.x] = (double)g;
    partials[stride + blockIdx.x] = (double)aleft;
  }
  if (last_cta(&u.cnt, u.ntile)) {
    if (threadIdx.x == 0) {
      double bg = 1e300;
      int al = 1;
      for (int i = 0; i < u.ntile; ++i) {
        const double pg = __ldcg(partials + u.tile0 + i);
        if (pg < bg) { bg = pg; al = (int)__ldcg(partials + stride + u.tile0 + i); }
      }
      const int64_t cut_a = u.cut[ca], cut_b = u.cut[cb];
      bool b_wins;
      if (cut_b != cut_a) b_wins = cut_b < cut_a;
      else b_wins = (bg < 1e300) && !al;  // equal cuts: the left set holding the smallest
                                          // differing gid wins (identical splits keep a)
      if (b_wins) u.best = cb;
    }
  }
}

int launch_choose(const LevelGraph& G, const Tile* tiles, int ntiles, Unit* units,
                  const uint64_t* ckey, const uint8_t* side, int cb, double* partials,
                  cudaStream_t s) {
  if (ntiles <= 0) return RSB_OK;
  k_choose<<<ntiles, RSB_BLOCK, 0, s>>>(G.gid, tiles, units, ckey, side, cb, partials, ntiles);
  RSB_CKL("k_choose");
  return RSB_OK;
}

// ----------------------------------------------------------------------------
// final side of every row of the level (0 left, 1 right)
// ----------------------------------------------------------------------------
// seg_split[s]: 1 when segment s is bisected at this level.
// seg_keystar[s]: component key of the straddling (or last fitting) component.
// seg_unit[s]: unit solving the straddler, or -1 when components fit exactly.
__global__ void k_finalize_side(const int32_t* __restrict__ row_seg, int32_t n,
                                const uint8_t* __restrict__ seg_split,
                                const uint64_t* __restrict__ seg_keystar,
                                const int32_t* __restrict__ seg_unit, const Unit* units,
                                const uint64_t* __restrict__ ckey, uint8_t* side) {
  const int r = blockIdx.x * RSB_BLOCK + threadIdx.x;
  if (r >= n) return;
  const int s = row_seg[r];
  uint8_t out = 0;
  if (seg_split[s]) {
    const uint64_t k = ckey[r], ks = seg_keystar[s];
    if (k < ks) out = 0;
    else if (k > ks) out = 1;
    else {
      const int ui = seg_unit[s];
      out = ui < 0 ? 0 : (uint8_t)((side[r] >> units[ui].best) & 1);
    }
  }
  side[r] = out;
}

int launch_finalize_side(const LevelGraph& G, const uint8_t* seg_split,
                         const uint64_t* seg_keystar, const int32_t* seg_unit, const Unit* units,
                         const uint64_t* ckey, uint8_t* side, cudaStream_t s) {
  if (G.n <= 0) return RSB_OK;
  k_finalize_side<<<(G.n + RSB_BLOCK - 1) / RSB_BLOCK, RSB_BLOCK, 0, s>>>(
      G.row_seg, G.n, seg_split, seg_keystar, seg_unit, units, ckey, side);
  RSB_CKL("k_finalize_side");
  return RSB_OK;
}
