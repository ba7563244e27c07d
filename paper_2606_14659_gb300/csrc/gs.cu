// gs.cu — the element dual graph from element -> vertex ids, and the Laplacian
// action without a stored graph (paper §5, gather-scatter; §2, weights).
//
// Input: ne elements, nv global vertex ids each (8 for hexes), ids in
// [0, V).  Set-up: the elements at every global vertex ("buckets": a
// counting sort by vertex id, then every bucket sorted by element id, so the
// result does not depend on the order of the atomics).  Q^T of §5 is then a
// sum over a bucket, Q a read of the vertex's sum.
//   * dual graph: element e's neighbours are the other elements in the buckets
//     of its vertices; the weight of neighbour f is how many of e's vertices f
//     shares (omega of §2): one pass counts the distinct neighbours (row
//     lengths), a scan gives row_ptr, a second pass writes them in ascending
//     order;
//   * matrix-free action y = (D_w - A_w) x with A_w = P^T Q Q^T P: per vertex
//     w_v = sum of x over its bucket (Q^T P x), per element
//     y_e = sum over e's vertices v of (c_v x_e - w_v), c_v the bucket size,
//     which is sum_v sum_{f at v} (x_e - x_f): the diagonal term of A_w and
//     D_w cancel inside every vertex term.
#include "rsb_internal.cuh"

#define GS_MAXCAND 256  // neighbour candidates of one element (with repeats)

__global__ void k_gs_maxid(const int64_t* __restrict__ ev, int64_t cnt, unsigned long long* vmax,
                           int* flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  long long m = -1;
  if (i < cnt) {
    m = ev[i];
    if (m < 0 || m >= (1ll << 31)) {
      atomicOr(flag, 1);
      m = -1;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m >= 0) atomicMax(vmax, (unsigned long long)m);
}

__global__ void k_gs_count(const int64_t* __restrict__ ev, int64_t cnt, int64_t* count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) atomicAdd((unsigned long long*)(count + ev[i]), 1ull);
}

// bucket fill (element ids; within a bucket in arrival order) and the slot
// table ev32 (vertex ids as int32)
__global__ void k_gs_fill(const int64_t* __restrict__ ev, int64_t cnt, int nv,
                          const int64_t* __restrict__ bptr, int64_t* cursor, int32_t* bucket,
                          int32_t* ev32) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  const int64_t v = ev[i];
  const unsigned long long pos = atomicAdd((unsigned long long*)(cursor + v), 1ull);
  bucket[bptr[v] + (int64_t)pos] = (int32_t)(i / nv);
  ev32[i] = (int32_t)v;
}

// every bucket sorted by element id (insertion sort: buckets are small)
__global__ void k_gs_sort(const int64_t* __restrict__ bptr, int64_t V, int32_t* bucket) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const int64_t b = bptr[v], e = bptr[v + 1];
  for (int64_t p = b + 1; p < e; ++p) {
    const int32_t x = bucket[p];
    int64_t q = p - 1;
    while (q >= b && bucket[q] > x) {
      bucket[q + 1] = bucket[q];
      --q;
    }
    bucket[q + 1] = x;
  }
}

// Distinct neighbours of element e with their shared-vertex counts, ascending;
// returns their number (or -1 when the candidates overflow GS_MAXCAND).
__device__ int gs_neighbours(int64_t e, int nv, const int32_t* __restrict__ ev32,
                             const int64_t* __restrict__ bptr, const int32_t* __restrict__ bucket,
                             int32_t* cand) {
  int nc = 0;
  for (int a = 0; a < nv; ++a) {
    const int32_t v = ev32[e * nv + a];
    for (int64_t p = bptr[v]; p < bptr[v + 1]; ++p) {
      const int32_t f = bucket[p];
      if (f == (int32_t)e) continue;
      if (nc >= GS_MAXCAND) return -1;
      cand[nc++] = f;
    }
  }
  for (int p = 1; p < nc; ++p) {  // insertion sort
    const int32_t x = cand[p];
    int q = p - 1;
    while (q >= 0 && cand[q] > x) {
      cand[q + 1] = cand[q];
      --q;
    }
    cand[q + 1] = x;
  }
  return nc;
}

__global__ void k_gs_rowlen(int64_t ne, int nv, const int32_t* __restrict__ ev32,
                            const int64_t* __restrict__ bptr, const int32_t* __restrict__ bucket,
                            int64_t* len, int* flag) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  int32_t cand[GS_MAXCAND];
  const int nc = gs_neighbours(e, nv, ev32, bptr, bucket, cand);
  if (nc < 0) {
    atomicOr(flag, 2);
    len[e] = 0;
    return;
  }
  int64_t d = 0;
  int run = 0;
  for (int p = 0; p < nc; ++p) {
    run = (p > 0 && cand[p] == cand[p - 1]) ? run + 1 : 1;
    if (p + 1 == nc || cand[p + 1] != cand[p]) {
      ++d;
      if (run > 7) atomicOr(flag, 4);  // more than 7 shared vertices: duplicate elements
    }
  }
  len[e] = d;
}

__global__ void k_gs_dual(int64_t ne, int nv, const int32_t* __restrict__ ev32,
                          const int64_t* __restrict__ bptr, const int32_t* __restrict__ bucket,
                          const int64_t* __restrict__ row_ptr, int32_t* col, int32_t* wt) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  int32_t cand[GS_MAXCAND];
  const int nc = gs_neighbours(e, nv, ev32, bptr, bucket, cand);
  if (nc < 0) return;
  int64_t out = row_ptr[e];
  int run = 0;
  for (int p = 0; p < nc; ++p) {
    run = (p > 0 && cand[p] == cand[p - 1]) ? run + 1 : 1;
    if (p + 1 == nc || cand[p + 1] != cand[p]) {
      col[out] = cand[p];
      wt[out] = run;
      ++out;
    }
  }
}

// w_v = sum of x over the elements at vertex v (Q^T P x), in bucket order
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_gs_vsum(int64_t nvert, const int64_t* __restrict__ bptr,
                                                     const int32_t* __restrict__ bucket,
                                                     const V* __restrict__ x, V* w) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvert) return;
  const int64_t b = bptr[v], e = bptr[v + 1];
  V s = V(0);
  for (int64_t p = b; p < e; ++p) s += __ldg(x + bucket[p]);
  w[v] = s;
}

// y_e = sum over e's vertices of (c_v x_e - w_v): (D_w - A_w) x, no stored graph
template <typename V>
__global__ void __launch_bounds__(RSB_BLOCK) k_gs_apply(int64_t ne, int nv,
                                                      const int32_t* __restrict__ ev32,
                                                      const int64_t* __restrict__ bptr,
                                                      const V* __restrict__ w,
                                                      const V* __restrict__ x, V* y) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const V xe = x[e];
  V acc = V(0);
  for (int a = 0; a < nv; ++a) {
    const int32_t v = __ldg(ev32 + e * nv + a);
    const V c = V(__ldg(bptr + v + 1) - __ldg(bptr + v));
    acc += c * xe - __ldg(w + v);
  }
  y[e] = acc;
}

// ----------------------------------------------------------------------------
// launchers (workspace: the caller's; sizes from gs_sizes)
// ----------------------------------------------------------------------------
static unsigned grid_of(int64_t n, int block = RSB_BLOCK) {
  return (unsigned)((n + block - 1) / block);
}

// Largest vertex id + 1 (V) of the table, or an error for ids outside [0, 2^31).
int gs_vertex_count(const int64_t* ev, int64_t cnt, unsigned long long* d_vmax, int* d_flag,
                    int64_t* V, cudaStream_t s) {
  RSB_CK(cudaMemsetAsync(d_vmax, 0, sizeof(unsigned long long), s));
  RSB_CK(cudaMemsetAsync(d_flag, 0, sizeof(int), s));
  if (cnt > 0) {
    k_gs_maxid<<<grid_of(cnt), RSB_BLOCK, 0, s>>>(ev, cnt, d_vmax, d_flag);
    RSB_CKL("k_gs_maxid");
  }
  unsigned long long vm = 0;
  int fl = 0;
  RSB_CK(cudaMemcpyAsync(&vm, d_vmax, sizeof(vm), cudaMemcpyDeviceToHost, s));
  RSB_CK(cudaMemcpyAsync(&fl, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  RSB_CK(cudaStreamSynchronize(s));
  if (fl) return rsb_set_error(RSB_EINVAL, "vertex ids must lie in [0, 2^31)");
  *V = cnt > 0 ? (int64_t)vm + 1 : 0;
  return RSB_OK;
}

// Buckets: bptr[V + 1], bucket[ne * nv], ev32[ne * nv]; count and cursor are
// int64[V + 1] scratch.
int gs_buckets(const int64_t* ev, int64_t ne, int nv, int64_t V, int64_t* count, int64_t* cursor,
               int64_t* bptr, int32_t* bucket, int32_t* ev32, void* scan_tmp, size_t scan_bytes,
               cudaStream_t s) {
  const int64_t cnt = ne * nv;
  RSB_CK(cudaMemsetAsync(count, 0, sizeof(int64_t) * (size_t)(V + 1), s));
  RSB_CK(cudaMemsetAsync(cursor, 0, sizeof(int64_t) * (size_t)(V + 1), s));
  if (cnt > 0) {
    k_gs_count<<<grid_of(cnt), RSB_BLOCK, 0, s>>>(ev, cnt, count);
    RSB_CKL("k_gs_count");
  }
  int rc = launch_scan_i64(count, bptr, V + 1, scan_tmp, scan_bytes, s);
  if (rc) return rc;
  if (cnt > 0) {
    k_gs_fill<<<grid_of(cnt), RSB_BLOCK, 0, s>>>(ev, cnt, nv, bptr, cursor, bucket, ev32);
    RSB_CKL("k_gs_fill");
    k_gs_sort<<<grid_of(V), RSB_BLOCK, 0, s>>>(bptr, V, bucket);
    RSB_CKL("k_gs_sort");
  }
  return RSB_OK;
}

int gs_row_lengths(int64_t ne, int nv, const int32_t* ev32, const int64_t* bptr,
                   const int32_t* bucket, int64_t* len, int* d_flag, cudaStream_t s) {
  RSB_CK(cudaMemsetAsync(d_flag, 0, sizeof(int), s));
  if (ne <= 0) return RSB_OK;
  k_gs_rowlen<<<grid_of(ne, 128), 128, 0, s>>>(ne, nv, ev32, bptr, bucket, len, d_flag);
  RSB_CKL("k_gs_rowlen");
  return RSB_OK;
}

int gs_fill_dual(int64_t ne, int nv, const int32_t* ev32, const int64_t* bptr,
                 const int32_t* bucket, const int64_t* row_ptr, int32_t* col, int32_t* wt,
                 cudaStream_t s) {
  if (ne <= 0) return RSB_OK;
  k_gs_dual<<<grid_of(ne, 128), 128, 0, s>>>(ne, nv, ev32, bptr, bucket, row_ptr, col, wt);
  RSB_CKL("k_gs_dual");
  return RSB_OK;
}

int gs_apply(int f32, int64_t ne, int nv, int64_t V, const int32_t* ev32, const int64_t* bptr,
             const int32_t* bucket, const void* x, void* w, void* y, cudaStream_t s) {
  if (ne <= 0) return RSB_OK;
  if (f32) {
    k_gs_vsum<float><<<grid_of(V), RSB_BLOCK, 0, s>>>(V, bptr, bucket, (const float*)x, (float*)w);
    RSB_CKL("k_gs_vsum<f32>");
    k_gs_apply<float><<<grid_of(ne), RSB_BLOCK, 0, s>>>(ne, nv, ev32, bptr, (const float*)w,
                                                        (const float*)x, (float*)y);
    RSB_CKL("k_gs_apply<f32>");
  } else {
    k_gs_vsum<double><<<grid_of(V), RSB_BLOCK, 0, s>>>(V, bptr, bucket, (const double*)x,
                                                       (double*)w);
    RSB_CKL("k_gs_vsum<f64>");
    k_gs_apply<double><<<grid_of(ne), RSB_BLOCK, 0, s>>>(ne, nv, ev32, bptr, (const double*)w,
                                                         (const double*)x, (double*)y);
    RSB_CKL("k_gs_apply<f64>");
  }
  return RSB_OK;
}
