/*
 * rsb.h — C ABI of librsb: Recursive Spectral Bisection of element dual graphs
 * on one GPU (sm_103a).
 *
 * Method (Ratnayaka & Fischer, "parRSB: Exascale Spectral Element Mesh
 * Partitioning"):
 *   - the problem statement (§2): a graph G(V, E) with positive edge weights
 *     and a part count P; find disjoint V_1..V_P covering V whose sizes differ
 *     by at most one (the printed "= 1" is read as "<= 1");
 *   - the weighted Laplacian L = D - A (§4) and its action (§5, assembled form);
 *   - the Fiedler vector (§4, Eqs. eigen0/eigen1) by restarted Lanczos (§6)
 *     or by inverse iteration with CG (§7, Algorithm 2);
 *   - Recursive Spectral Bisection (§4, Algorithm 1) with floor/ceil splits of
 *     the part count and proportional element counts.
 *
 * Memory.  Every pointer argument may be a device pointer or a host pointer;
 * the library asks the CUDA runtime which it is.  Host inputs are copied to
 * the device and host outputs copied back inside the call (the call then
 * returns only after the copy-back).  The caller owns every buffer it passes;
 * the library keeps none of them after returning.  The library owns a cached
 * device workspace that grows as needed and is freed by rsb_release().
 *
 * Streams.  `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 * issued on that stream; the calls synchronise with it before returning
 * (convergence decisions and statistics are read back on the host).
 *
 * Errors.  Every call returns one of the RSB_* codes below; RSB_OK is 0.
 * Invalid arguments are rejected with RSB_EINVAL before any device work.
 * A device error is reported as RSB_ECUDA (the CUDA error string is kept for
 * rsb_last_error_detail()).  RSB_ENOCONV means some solve hit its iteration
 * cap; outputs are still written from the best iterate.
 *
 * Threading.  Calls are not re-entrant: one call at a time per process.
 */
#ifndef RSB_H
#define RSB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  RSB_OK = 0,
  RSB_EINVAL = 1,        /* bad argument or malformed graph                    */
  RSB_ENOMEM = 2,        /* device allocation failed                           */
  RSB_ECUDA = 3,         /* CUDA runtime / kernel error                        */
  RSB_ENOCONV = 4,       /* a Fiedler solve stopped at its iteration cap       */
  RSB_ETIMEOUT = 5,      /* a bounded device wait gave up                      */
  RSB_EDISCONNECTED = 6  /* rsb_fiedler: the graph has several components      */
};

enum { RSB_LANCZOS = 0, RSB_INVERSE = 1, RSB_RCB = 2 }; /* §6, §7; RCB of §5/§8 */
enum { RSB_FP64 = 0, RSB_MIXED = 1 };               /* arithmetic of the solves  */
enum { RSB_DEGEN_NONE = 0, RSB_DEGEN_RESOLVE = 1 }; /* repeated lambda_2 (§9)    */

/*
 * Symmetric graph in CSR form (the dual graph of §2).
 *   n        number of vertices (elements), 0 <= n < 2^29
 *   row_ptr  int64[n + 1], row_ptr[0] = 0, non-decreasing
 *   col      int32[row_ptr[n]], neighbour indices in [0, n), no self loops;
 *            the pattern and the weights must be symmetric
 *   weight   int32[row_ptr[n]], integer weights in 1..7 (the paper's weights
 *            are 1, 2, 4 shared vertices); NULL means every weight is 1
 *   gid      int64[n], global element ids used for tie-breaks and start
 *            vectors, distinct within one graph; NULL means gid = row index
 *   coords   double[3 n], (x, y, z) of every element (e.g. its centroid), row
 *            by row; needed only by method RSB_RCB and by reorder = 1, else
 *            may be NULL
 */
typedef struct rsb_csr {
  int64_t n;
  const int64_t *row_ptr;
  const int32_t *col;
  const int32_t *weight;
  const int64_t *gid;
  const double *coords;
} rsb_csr;

typedef struct rsb_options {
  int method;            /* RSB_LANCZOS | RSB_INVERSE: the Fiedler vector (§6, §7);
                            RSB_RCB: recursive coordinate bisection instead (the
                            geometric partitioner §5 and §8 run before RSB): every
                            segment splits along the axis of its largest coordinate
                            extent, lower coordinates left, ties by gid; needs
                            coords                                                  */
  int precision;         /* RSB_FP64 | RSB_MIXED (FP32 vectors + FP64 polish)      */
  int krylov_dim;        /* Lanczos steps per cycle, 2..40                         */
  int max_restarts;      /* Lanczos cycles per solve (paper §8: 50)                */
  double tol;            /* stop when ||L y - theta y|| <= tol * max weighted degree */
  double cg_tol;         /* CG stop: ||r|| <= cg_tol * ||b||                        */
  int cg_maxit;          /* CG iterations per outer step                           */
  int max_outer;         /* inverse-iteration outer steps                          */
  uint64_t seed;         /* start-vector seed                                      */
  int degenerate_policy; /* RSB_DEGEN_NONE | RSB_DEGEN_RESOLVE                     */
  double cluster_tol;    /* RESOLVE: |lambda_b - lambda_a| <= cluster_tol lambda_a  */
  double tie_rel;        /* median-split tie window, relative to the value range   */
  double mixed_tol;      /* MIXED: FP32 stage stops at max(tol, mixed_tol)         */
  int batched;           /* 1: all subgraphs of a level in one set of launches     */
  int use_graph;         /* launch mode of a Lanczos cycle: 0 one launch per kernel,
                            1 one CUDA graph per cycle, 2 one persistent cooperative
                            kernel per cycle, 3 one persistent cooperative kernel per
                            solve whose CTAs keep their tile's basis rows in shared
                            memory when every tile gets a co-resident CTA (else 1);
                            CG blocks use a CUDA graph for 1, 2 and 3                */
  int validate;          /* 1: also check symmetry of the input on the device      */
  int polish_cycles;     /* MIXED: at most this many FP64 Lanczos cycles of polish_dim
                            steps after the FP32 stage, stopping early at tol (0: only
                            the FP64 Rayleigh-quotient refinement of the FP32 vector) */
  int keep;              /* Ritz vectors kept by a thick restart, 0..16 (0: restart
                            from the Ritz vector alone)                               */
  int tile_rows;         /* rows per thread of a solver tile (a tile is 256 x this
                            many rows of one subgraph), 1..64; 0: the default 2     */
  int polish_dim;        /* MIXED: Lanczos steps per FP64 polish cycle, 2..40      */
  int block;             /* Lanczos block width, 1..4: 1 the single-vector method of
                            §6; 2..4 thick-restarted block Lanczos (the block
                            extension of §9) for every subgraph with at least
                            krylov_dim + block dimensions orthogonal to the fixed
                            basis, single-vector for smaller ones                  */
  int reorder;           /* 1: before the spectral recursion, order every mesh's
                            elements by recursive coordinate bisection into leaves
                            of 512..1023 elements (the RCB pre-partition of §5/§8;
                            on one GPU it makes the Laplacian's gathers local);
                            part ids are still returned in caller order; needs
                            coords.  0: keep the caller's order                    */
  int amg;               /* RSB_INVERSE: 1 solves L x = b by flexible CG
                            preconditioned with an aggregation AMG V-cycle (§7,
                            Algorithm 3; pairs of consecutive rows, RCB order with
                            reorder = 1); 0 plain CG                               */
} rsb_options;

typedef struct rsb_stats {
  int levels;                 /* bisection levels run                              */
  int nonconverged;           /* solves that stopped at their cap                  */
  int64_t solves;             /* Fiedler solves (units x candidates x precisions)  */
  int64_t cycles;             /* Lanczos cycles or inverse-iteration outer steps  */
  int64_t inner;              /* CG iterations (inverse iteration)                 */
  int64_t elements_bisected;  /* sum over levels and split segments of their size */
  double lambda_first;        /* lambda_2 of the first split of the first mesh     */
  double resid_max;           /* largest final ||L y - theta y|| / max degree      */
  double seconds;             /* wall time of the call, host clock                 */
  int64_t kernel_launches;    /* kernels issued by the call                        */
} rsb_stats;

/* Fills *o with the defaults: Lanczos, FP64, krylov_dim 40, max_restarts 50,
 * tol 1e-10, cg_tol 1e-12, cg_maxit 4000, max_outer 50, RESOLVE,
 * cluster_tol 0.05, tie_rel 1e-5, mixed_tol 1e-6, batched 1, use_graph 3,
 * validate 0, polish_cycles 2, keep 8, tile_rows 0, polish_dim 16, block 1,
 * reorder 0, amg 0. */
void rsb_options_default(rsb_options *o);

/*
 * Recursive spectral bisection of one graph into nparts parts (§4,
 * Algorithm 1; sizes per §4: a segment of parts [p0, p1) holds
 * floor(p1 n / P) - floor(p0 n / P) elements and its left child gets the
 * floor((p1 - p0) / 2) lower-numbered parts).
 *   g       the graph (device or host pointers)
 *   nparts  1 <= nparts <= n
 *   o       options (NULL = defaults)
 *   part    int32[n] output, part id of every row in [0, nparts)
 *   st      optional statistics (host pointer, may be NULL)
 * Returns RSB_EINVAL for nparts out of range or a malformed graph.
 */
int rsb_partition(const rsb_csr *g, int32_t nparts, const rsb_options *o,
                  int32_t *part, rsb_stats *st, void *stream);

/*
 * rsb_partition for nmesh independent graphs at once: every bisection level of
 * every mesh is solved together (one set of launches per level when
 * o->batched).  gs[m], nparts[m] and parts[m] are the arguments of mesh m
 * (host arrays of structs/pointers; the pointers inside may be device or
 * host).  Results equal nmesh separate rsb_partition calls.
 */
int rsb_partition_batch(const rsb_csr *gs, int32_t nmesh, const int32_t *nparts,
                        const rsb_options *o, int32_t *const *parts, rsb_stats *st,
                        void *stream);

/*
 * rsb_autotune: picks the tile rows (2, 4 or 8 rows per thread; a solver tile
 * is 256 x that many rows of one subgraph) and the launch mode of the Lanczos
 * cycles (3 or 1, see use_graph) for a workload by timing it.  Each of the
 * RSB_TUNE_CANDIDATES candidates, in the order (2,3) (4,3) (8,3) (2,1) (4,1)
 * (8,1) of (tile_rows, use_graph), runs one bisection level of the given meshes
 * with two Lanczos cycles, no polish and no deflated candidates, once untimed
 * and twice timed with CUDA events on the stream; the fastest is written into
 * o->tile_rows and o->use_graph, every other field of *o is kept.  Launch
 * modes give identical results; tile rows change the order of the reductions'
 * partial sums (rounding only).
 *   gs, nmesh, nparts, parts  as in rsb_partition_batch; parts[m] is
 *           overwritten (scratch)
 *   o       in: the options of the real run; out: with the chosen tile_rows
 *           and use_graph (host pointer, not NULL)
 *   ms_out  optional host array of RSB_TUNE_CANDIDATES doubles: the best time
 *           of each candidate in ms
 * The call synchronises the stream.  Returns the first error of a candidate
 * run (RSB_ENOCONV of the two-cycle runs is expected and ignored).
 */
#define RSB_TUNE_CANDIDATES 6
int rsb_autotune(const rsb_csr *gs, int32_t nmesh, const int32_t *nparts, rsb_options *o,
                 int32_t *const *parts, double *ms_out, void *stream);

/*
 * Fiedler pair of a connected graph (§4, Eqs. eigen0/eigen1; §6 or §7).
 *   lambda2  host double out: the smallest eigenvalue of L on 1-perp
 *   v        double[n] out: unit Fiedler vector, sign fixed so that the
 *            smallest gid among |v_i| >= max|v| / 2 has v_i < 0
 *   resid    host double out (nullable): ||L v - lambda2 v||_2
 * With several components returns RSB_EDISCONNECTED, lambda2 = 0 and v the
 * normalised contrast vector of the component holding the smallest gid
 * against the rest.  n must be >= 2.
 */
int rsb_fiedler(const rsb_csr *g, const rsb_options *o, double *lambda2, double *v,
                double *resid, void *stream);

/*
 * y = L x with L = D - A of graph g (§4 weighted Laplacian, §5 action), on the
 * library's sliced-ELL form, in FP64 (x, y double[n]) or FP32 (x, y float[n]).
 * A building block exposed for testing and bandwidth measurement.
 */
int rsb_laplacian_apply(const rsb_csr *g, const double *x, double *y, void *stream);
int rsb_laplacian_apply_f32(const rsb_csr *g, const float *x, float *y, void *stream);

/*
 * Times `reps` back-to-back applications of the sliced-ELL Laplacian kernel
 * (FP64 when f32 == 0, else FP32) on graph g with CUDA events on `stream`;
 * *ms_per_apply receives the mean device time of one launch and
 * *useful_bytes the algorithmic bytes of one launch (4 B per stored entry
 * plus one read of x and one write of y).  Build time is excluded.
 */
int rsb_laplacian_bench(const rsb_csr *g, int f32, int reps, double *ms_per_apply,
                        double *useful_bytes, void *stream);

/*
 * The element dual graph of a mesh given as element -> global vertex ids
 * (§2: elements are adjacent when they share a vertex, the weight omega is the
 * number of shared vertices; §5: the same graph is P^T Q Q^T P without its
 * diagonal).  Built on the GPU: the elements at every vertex are collected
 * (a counting sort by vertex id), then every element's distinct neighbours
 * are counted and written in ascending order.
 *   ne       number of elements, 1 <= ne < 2^29
 *   nv       vertices per element, 1..8 (8 for hexes)
 *   ev       int64[ne * nv], the vertex ids of element e at ev[e*nv .. e*nv+nv-1],
 *            each in [0, 2^31)
 *   row_ptr  int64[ne + 1] out (device or host)
 *   col, weight  int32[cap] out, or both NULL to learn nnz first
 *   cap      room in col and weight
 *   nnz      host int64 out: the number of stored entries
 * Rows list columns in ascending order with weights 1..7 (the CSR rsb_partition
 * takes).  RSB_EINVAL for ids outside [0, 2^31), an element meeting more than
 * 256 others at its vertices, two elements sharing more than 7 vertices, or
 * cap < nnz (row_ptr and nnz are still written then).
 */
int rsb_dual_graph(int64_t ne, int nv, const int64_t *ev, int64_t *row_ptr, int32_t *col,
                   int32_t *weight, int64_t cap, int64_t *nnz, void *stream);

/*
 * y = L x without a stored graph: the gather-scatter form of §5,
 * L = D_w - A_w with A_w = P^T Q Q^T P.  Every element's value is summed per
 * global vertex (Q^T P x), and element e collects sum over its vertices v of
 * (c_v x_e - w_v), c_v the number of elements at v and w_v their sum: the
 * weighted Laplacian of the dual graph above.  ne, nv, ev as in
 * rsb_dual_graph; x, y double[ne] (or float[ne] for the _f32 form), device or
 * host.  The vertex buckets are rebuilt by every call.
 */
int rsb_laplacian_apply_gs(int64_t ne, int nv, const int64_t *ev, const double *x, double *y,
                           void *stream);
int rsb_laplacian_apply_gs_f32(int64_t ne, int nv, const int64_t *ev, const float *x, float *y,
                               void *stream);

/*
 * Times `reps` gather-scatter Laplacian applications (two kernels each; FP64
 * when f32 == 0) after building the vertex buckets once; *ms_per_apply gets
 * the mean device time of one application, *useful_bytes its algorithmic
 * bytes (bucket offsets twice, the bucket entries and vertex ids once each,
 * x read once, the vertex sums written and read once, y written once).
 */
int rsb_laplacian_bench_gs(int64_t ne, int nv, const int64_t *ev, int f32, int reps,
                           double *ms_per_apply, double *useful_bytes, void *stream);

/*
 * rsb_laplacian_apply_noalloc — y = L x (FP64) like rsb_laplacian_apply, for
 * callers that cannot allocate device memory.  The paper has no counterpart;
 * this is a deployment variant.  Some callers must not call cudaMalloc: code
 * running while a framework's caching allocator holds the whole device, code
 * in a region where the implicit synchronisation of cudaMalloc/cudaFree is not
 * allowed, or embedders that budget every device byte up front.  This call
 * allocates nothing: its scratch (the sliced-ELL copy of g and a scan
 * workspace) lives in one 32 MiB device array compiled into the library, which
 * every GPU that loads the library holds until the process exits.
 *   g, x, y  device pointers only (RSB_EINVAL otherwise); x, y double[n]
 *   stream   used directly; the call returns after the result is on it
 * Graphs whose scratch exceeds the 32 MiB (4 B per padded SELL entry plus
 * about 5 B per row) are rejected with RSB_EINVAL.  All calls share the array
 * and leave their contents in it; each call clears what must start at zero.
 * Calls that overlap on the GPU (other streams or host threads) race on the
 * array: order them.  Every call reads the entry count back to the host and
 * synchronises `stream`, so it cannot be used inside a stream capture.  The
 * first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it.
 */
int rsb_laplacian_apply_noalloc(const rsb_csr *g, const double *x, double *y, void *stream);

/* Static description of an error code. */
const char *rsb_strerror(int code);

/* Detail of the last RSB_ECUDA / RSB_EINVAL error (thread-unsafe). */
const char *rsb_last_error_detail(void);

/* Frees the cached device workspace (all devices touched by this process). */
void rsb_release(void);

#ifdef __cplusplus
}
#endif

#endif /* RSB_H */
