/* cudapre.h -- C ABI of the GB300 (sm_103a) implementation of the CudaPre
 * convex-hull preprocessing method: G. Mei, "A Straightforward Preprocessing
 * Approach for Accelerating Convex Hull Computations on the GPU",
 * arXiv 1405.3454.
 *
 * The method (section 2):
 *   Step 1  16 extreme points: min/max of x and y in the original point set
 *           and in three rotated copies of it;
 *   Step 2  the convex polygon of those points by Andrew's monotone chain
 *           (the paper's correction note: reference [6] is Andrew's algorithm);
 *   Step 3  discard every point strictly inside that polygon;
 *   then    the convex hull of the remaining points (section 3, case (2)).
 * Every step runs on the GPU; the host only enqueues work.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Points     float32 xy interleaved, point i at xy[2i], xy[2i+1].  The
 *            address must be 8-byte aligned.  Coordinates must be finite,
 *            integer-valued and within [-2^24, 2^24]; then every orientation
 *            test is exact in int64 and every result is bit-exact.  Outside
 *            that domain results are undefined unless options.validate is set,
 *            in which case the call flags HULL_DEVICE_DOMAIN (see
 *            hull_get_device_status) and produces empty results.
 * Rotations  counter-clockwise, x' = x c - y s, y' = x s + y c, evaluated as
 *            RN(RN(x*c) - RN(y*s)) and RN(RN(x*s) + RN(y*c)) in binary64 with
 *            c, s the correctly rounded closed forms.  Ties go to the lowest
 *            index.
 * Extremes   16 slots, slot 4g+k for rotation group g (0 = original set) and
 *            k = 0 argmin x', 1 argmax x', 2 argmin y', 3 argmax y'.
 * Inside     strictly inside: points on the polygon boundary remain.  A
 *            polygon with fewer than 3 vertices discards nothing.
 * Hull       strictly convex (collinear boundary points are not vertices),
 *            counter-clockwise from the lexicographically smallest (x, y)
 *            vertex; among equal coordinates the lowest index is reported.
 * Memory     the caller owns every buffer (inputs, outputs, workspace), all in
 *            device memory unless stated.  The library allocates nothing.
 * Streams    `stream` is a cudaStream_t (NULL = the legacy default stream).
 *            Calls are asynchronous: they return after enqueueing.  Counts
 *            are written to device memory.  A workspace must not be shared by
 *            calls that may overlap on the GPU; distinct workspaces are
 *            independent and may be used from different host threads.
 * Errors     the return value reports argument and launch errors; conditions
 *            found on the device are recorded in the workspace and read with
 *            hull_get_device_status.
 */
#ifndef CUDAPRE_H
#define CUDAPRE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum hull_status {
  HULL_OK = 0,
  HULL_ERR_INVALID_ARG = 1, /* null pointer, negative or too large size, misalignment */
  HULL_ERR_DOMAIN = 2,      /* reported by hull_get_device_status: input outside the domain */
  HULL_ERR_WORKSPACE = 3,   /* workspace smaller than the matching *_workspace_bytes */
  HULL_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed */
  HULL_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  HULL_ERR_BUDGET = 6,      /* request larger than the configured memory budget */
  HULL_ERR_UNSUPPORTED = 7  /* option value not supported */
} hull_status;

/* Angle tables for Step 1 (section 2).  CUMULATIVE reads "rotate in 30, 45
 * and 45 degrees" as 30, 75 and 120 degrees from the original set; ABSOLUTE
 * is the 30, 45, 60 degrees of Figure 1 and section 5. */
#define HULL_ANGLES_CUMULATIVE 0
#define HULL_ANGLES_ABSOLUTE 1

/* Arithmetic of the inside test and of the extreme search.
 * EXACT: binary64 projections for every point and an int64 orientation test
 *        for every edge -- the plain method.
 * FP32:  float32 projections and orientation tests with a static error
 *        bound; only decisions inside the bound are escalated to binary64 /
 *        int64.  Results are bit-identical to EXACT. */
#define HULL_FILTER_EXACT 0
#define HULL_FILTER_FP32 1

typedef struct hull_options {
  int32_t angles;        /* HULL_ANGLES_*; default CUMULATIVE */
  int32_t filter;        /* HULL_FILTER_*; default FP32 */
  int32_t validate;      /* nonzero: check the input domain on the device first */
  int32_t block;         /* threads per block of the streaming kernels; 0 = tuned */
  int32_t grid;          /* blocks of the streaming kernels; 0 = tuned */
  int32_t refine;        /* hull_compute: 1 (default) = a second, finer discard
                            round on the survivors before the final hull (same
                            result, less work); 0 = sort and chain every survivor */
  int32_t no_prefilter;  /* hull_compute: 0 (default) = the method; 1 = the hull of
                            all points without Steps 1-3 (the paper's case (1),
                            for comparison; same result).  Not for hull_prefilter
                            or a batch (HULL_ERR_UNSUPPORTED). */
  int32_t waves;         /* a batch's streaming extreme search: waves of resident
                            blocks its static shares make (1 .. 16); 0 = tuned */
  int32_t unit_chunks;   /* a batch's inside test: pairs claimed at a time, in
                            chunks of 1024 pairs (1 .. 1024); 0 = tuned.  No
                            launch-shape option changes any result. */
  int32_t reserved[7];   /* must be zero */
} hull_options;

/* Device-side condition bits (hull_get_device_status). */
#define HULL_DEVICE_DOMAIN 1u   /* validate found a coordinate outside the domain */
#define HULL_DEVICE_TIMEOUT 2u  /* a bounded wait expired */
#define HULL_DEVICE_OVERFLOW 4u /* an internal capacity was exceeded */
#define HULL_DEVICE_OFFSETS 8u  /* hull_batch: offsets[0] != 0, decreasing, offsets[S] != n_total,
                                   a set of 2^32 points or more, or a range beyond the pool */

/* Fills *opt with the defaults (cumulative angles, FP32 filter, no validation,
 * tuned launch shapes, refinement on). */
void hull_default_options(hull_options* opt);

/* Bytes of workspace needed by hull_prefilter for n points (opt may be NULL
 * for the defaults).  The workspace needs no initialisation. */
size_t hull_prefilter_workspace_bytes(int64_t n, const hull_options* opt);

/* Bytes of workspace needed by hull_compute for n points: about 24 bytes per
 * point plus 1.3 MB; from 2^24 points on, about 25 MB more (survivor slots
 * the inside test may reserve ahead). */
size_t hull_workspace_bytes(int64_t n, const hull_options* opt);

/* Steps 1-3 of section 2 on one point set.
 *   d_xy             n points (see Points above); n in [0, 2^32 - 1].
 *   d_ws, ws_bytes   workspace of at least hull_prefilter_workspace_bytes(n).
 *   d_survivor_idx   room for n uint32: indices of the points NOT strictly
 *                    inside the polygon of the extremes, in unspecified order
 *                    (compare as a set).
 *   d_n_survivors    one int64: the number of survivors.
 *   d_extreme_idx    16 uint32 (may be NULL): the extreme indices, see
 *                    Extremes above; all 0xFFFFFFFF when n == 0.
 * The polygon stays in the workspace (hull_read_polygon). */
hull_status hull_prefilter(const float* d_xy, int64_t n, void* d_ws, size_t ws_bytes,
                           uint32_t* d_survivor_idx, int64_t* d_n_survivors,
                           uint32_t* d_extreme_idx, const hull_options* opt, void* stream);

/* The whole method on one point set: Steps 1-3, compaction of the survivors,
 * then the hull of the survivors (section 3, case (2)): a second discard
 * round (option refine; points strictly inside triangles of farthest
 * survivors), then up to 8192 points a hull classified on the whole GPU,
 * more a device radix sort and Andrew's monotone chain.
 *   d_ws             at least hull_workspace_bytes(n).
 *   d_hull_idx       room for n uint32: hull vertex indices, see Hull above.
 *   d_n_hull         one int64: the number of hull vertices (0 when n == 0). */
hull_status hull_compute(const float* d_xy, int64_t n, void* d_ws, size_t ws_bytes,
                         uint32_t* d_hull_idx, int64_t* d_n_hull,
                         const hull_options* opt, void* stream);

/* Bytes of workspace needed by hull_batch for S sets of n_total points in
 * all: about 28 bytes per point plus about 0.25 MB per set. */
size_t hull_batch_workspace_bytes(int64_t n_total, int32_t S, const hull_options* opt);

/* The whole method (as hull_compute) on each of S point sets in one call.
 * Every step runs for all sets at once: the two streaming passes split the
 * concatenated points evenly over the GPU, the per-set steps run one block
 * (or a few) per set.
 *   d_xy             n_total points; set s is points [offsets[s], offsets[s+1]).
 *                    A set may start at any point (8-byte alignment).
 *   d_offsets        S+1 int64 in device memory: 0 = offsets[0] <= offsets[1]
 *                    <= ... <= offsets[S] = n_total; each set below 2^32
 *                    points.  Checked on the device: a violation records
 *                    HULL_DEVICE_OFFSETS and every set's hull is empty.
 *   S                number of sets, >= 0.
 *   n_total          offsets[S] as known to the caller (sizes the workspace).
 *   d_ws, ws_bytes   at least hull_batch_workspace_bytes(n_total, S).
 *   d_hull_idx       room for n_total int64: the hulls of all sets, set after
 *                    set, as GLOBAL point indices (offsets[s] + the index
 *                    within the set), each as described under Hull above.
 *   d_hull_offsets   S+1 int64: set s's hull is d_hull_idx[d_hull_offsets[s]
 *                    .. d_hull_offsets[s+1]).
 * Device-side conditions of any set (and HULL_DEVICE_OFFSETS) are or-ed into
 * the word hull_get_device_status reads from d_ws; then every hull is empty.
 * The stats and polygon readers do not apply to a batch workspace. */
hull_status hull_batch(const float* d_xy, const int64_t* d_offsets, int32_t S, int64_t n_total, void* d_ws,
                       size_t ws_bytes, int64_t* d_hull_idx, int64_t* d_hull_offsets,
                       const hull_options* opt, void* stream);

/* hull_batch on sets taken anywhere in a pool of points: set s is the
 * offsets[s+1] - offsets[s] points of d_xy starting at row d_starts[s]
 * (sets may overlap, repeat or come in any order; a set may start at any
 * row).  offsets (S+1, from 0 to n_total) then only give the sizes and the
 * order of the output; the workspace is hull_batch_workspace_bytes(n_total,
 * S).  Hull indices are rows of d_xy (d_starts[s] + the index within the
 * set).  d_starts (S int64, device) is checked on the device: a set beyond
 * the n_xy points records HULL_DEVICE_OFFSETS.  The paper has no
 * counterpart: it lets a server batch requests that point into a resident
 * pool without copying their points. */
hull_status hull_batch_ranges(const float* d_xy, int64_t n_xy, const int64_t* d_starts, const int64_t* d_offsets,
                              int32_t S, int64_t n_total, void* d_ws, size_t ws_bytes, int64_t* d_hull_idx,
                              int64_t* d_hull_offsets, const hull_options* opt, void* stream);

/* ---- Batches as CUDA graphs (the paper has no counterpart) ------------ */

/* A host object that runs hull_batch_ranges calls as CUDA graphs, so that a
 * repeated batch launches all of its kernels with one graph launch.  The
 * first call captures the call's work on `stream` into a graph and
 * instantiates it.  A call whose arguments and options all equal the
 * previous call's replays that graph (the kernels read every size, offset
 * and start from device memory, so new contents of the same buffers are
 * fine).  Any other call captures anew and updates the instantiated graph in
 * place, or instantiates a new one when CUDA refuses the update (another
 * sequence of kernels, e.g. other options).  Results, workspace sizes and
 * device-side status are those of hull_batch_ranges.
 *   stream   must not be the legacy default stream (NULL): it cannot be
 *            captured (HULL_ERR_INVALID_ARG); nor may it be capturing already.
 * Not thread-safe: one host thread per object; no stage timer may be
 * attached on that thread during a capture. */
typedef struct hull_graph hull_graph;
hull_graph* hull_graph_create(void);
void hull_graph_destroy(hull_graph* g);
hull_status hull_graph_batch_ranges(hull_graph* g, const float* d_xy, int64_t n_xy, const int64_t* d_starts,
                                    const int64_t* d_offsets, int32_t S, int64_t n_total, void* d_ws,
                                    size_t ws_bytes, int64_t* d_hull_idx, int64_t* d_hull_offsets,
                                    const hull_options* opt, void* stream);
/* h_out[6] (host): calls, captures, in-place updates, instantiations,
 * replays, and the kernels of the current graph. */
void hull_graph_counts(const hull_graph* g, int64_t* h_out);

/* hull_compute without a caller workspace; the paper has no counterpart (it
 * is a library convenience, not a step of the method).  The workspace is a
 * fixed device array inside the library (about 26 MiB per device, allocated
 * by the CUDA runtime when the library's module loads), so the call allocates
 * nothing.  It is meant for callers that cannot allocate: loops where
 * cudaMalloc / cudaFree would synchronise the device, or programs whose
 * device memory is already fully reserved.
 *   n                at most HULL_STATIC_MAX_POINTS; larger n returns
 *                    HULL_ERR_BUDGET before any CUDA call.
 *   d_hull_idx, d_n_hull, opt, stream   as for hull_compute.
 * The first call on a device looks up the array's device address (a runtime
 * query, not a stream operation); make it before any stream capture begins
 * on that device.  The address is kept for the life of the process: after
 * cudaDeviceReset on a device (which unloads the library's module there) do
 * not call this entry point on that device again.  The counters that must start at zero are cleared by every
 * call on its stream.  There is ONE such workspace per device: calls on the
 * same device that may overlap on the GPU (other streams, other host threads)
 * race on it and corrupt each other's results; order them on one stream.
 * hull_read_stats and the other readers take a workspace pointer and cannot
 * see this one. */
#define HULL_STATIC_MAX_POINTS 1048576
hull_status hull_compute_static(const float* d_xy, int64_t n, uint32_t* d_hull_idx, int64_t* d_n_hull,
                                const hull_options* opt, void* stream);

/* Number of survivors and of FP32 decisions escalated to the exact test by
 * the last hull_prefilter / hull_compute on this workspace.  Synchronises the
 * stream.  Either output pointer may be NULL (host memory). */
hull_status hull_read_counters(const void* d_ws, int64_t* h_n_survivors,
                               int64_t* h_n_escalated, void* stream);

/* Counters of the last hull_prefilter / hull_compute on a workspace. */
typedef struct hull_stats {
  int64_t n_survivors;      /* points not strictly inside the Step-2 polygon */
  int64_t n_escalated;      /* float32 decisions escalated to exact arithmetic */
  int64_t n_refined;        /* entries left by the refinement round (hull_compute); on one set
                               this can include copies of a survivor (same index), which
                               hull_compute's survivor buffer holds in reserved slots */
  int32_t polygon_vertices; /* vertices of the Step-2 polygon */
  uint32_t device_status;   /* HULL_DEVICE_* bits */
} hull_stats;

/* Reads the counters of the last call on this workspace (host memory);
 * synchronises the stream. */
hull_status hull_read_stats(const void* d_ws, hull_stats* h_out, void* stream);

/* The Step-2 polygon of the last call on this workspace: *h_m vertices,
 * h_xy[2k], h_xy[2k+1] their integer coordinates counter-clockwise from the
 * lexicographic minimum (room for 32 int32), h_idx[k] their point indices
 * (room for 16 uint32; may be NULL).  Synchronises the stream (host memory). */
hull_status hull_read_polygon(const void* d_ws, int32_t* h_m, int32_t* h_xy,
                              uint32_t* h_idx, void* stream);

/* One set of the last hull_batch / hull_batch_ranges call on a batch
 * workspace (host memory). */
typedef struct hull_set_info {
  int32_t polygon_vertices;   /* vertices of the set's Step-2 polygon */
  int32_t polygon_xy[32];     /* their integer coordinates, as hull_read_polygon */
  uint32_t polygon_idx[16];   /* their indices within the set */
  uint32_t extreme_idx[16];   /* the set's 16 extremes (Extremes above), indices
                                 within the set; 0xFFFFFFFF when the set is empty */
  int64_t n_survivors;        /* points of the set left by Step 3 */
  int64_t n_escalated;        /* its float32 decisions escalated to exact arithmetic */
  int64_t n_refined;          /* entries left by its refinement round */
  uint32_t device_status;     /* the set's HULL_DEVICE_* bits */
  uint32_t pad_;
} hull_set_info;

/* Reads set s (0 <= s < S) of the last batch call on d_ws, a workspace laid
 * out for (n_total, S) as hull_batch_workspace_bytes; synchronises the
 * stream.  A set whose steps were skipped (a device condition of the batch)
 * reads as empty. */
hull_status hull_batch_read_set(const void* d_ws, int64_t n_total, int32_t S, int32_t s, hull_set_info* h_out,
                                void* stream);

/* Device-side condition bits (HULL_DEVICE_*) recorded by the last call on this
 * workspace; synchronises the stream.  Returns HULL_OK when no bit is set,
 * else the matching error code. */
hull_status hull_get_device_status(const void* d_ws, uint32_t* h_bits, void* stream);

/* Human-readable name of a status code (static storage). */
const char* hull_strerror(hull_status s);

/* The projection constants this library uses: out[0..3] = sqrt(3)/2,
 * (sqrt(6)-sqrt(2))/4, (sqrt(6)+sqrt(2))/4, sqrt(2)/2 (host memory). */
void hull_constants(double* out);

/* ABI version of this header. */
int32_t hull_abi_version(void);

/* ---- The 3D extension (section 5) ------------------------------------- */

/* Section 5 sketches the method in 3D: six extremes (min/max of x, y, z) of
 * the point set and of copies rotated about one axis, the convex polyhedron
 * of those points, and the discard of the points strictly inside it.  Here
 * the axis is z and the rotations are Step 1's angle table (options.angles):
 * x' and y' as in 2D, z' = z.
 * Points     float32 xyz interleaved (point i at xyz[3i..3i+2]), the address
 *            16-byte aligned; coordinates finite, integer-valued, within
 *            [-2^19, 2^19], so every plane test is exact in int64.  Outside
 *            that domain results are undefined unless options.validate is
 *            set (HULL_DEVICE_DOMAIN, empty results).
 * Extremes   24 slots, slot 6g + k for rotation group g: k = 0 argmin x',
 *            1 argmax x', 2 argmin y', 3 argmax y', 4 argmin z', 5 argmax
 *            z'; ties go to the lowest index.
 * Polyhedron facet planes (Nx, Ny, Nz, d), int64: every extreme satisfies
 *            N.p <= d; each plane once, reduced (gcd of the four absolute
 *            values 1), in lexicographic order.  Fewer than four affinely
 *            independent extremes give no facet, and nothing is discarded.
 * Inside     strictly inside: N.p < d for every facet.
 * Options    angles, filter (EXACT: binary64 projections and int64 plane
 *            tests throughout; FP32: float32 filters with exact escalation,
 *            identical results) and validate apply; no_prefilter does not. */
#define HULL3_SLOTS 24
#define HULL3_MAX_FACETS 48

/* Bytes of workspace hull3_prefilter needs (a fixed 1.2 MB; n may be any). */
size_t hull3_prefilter_workspace_bytes(int64_t n, const hull_options* opt);

/* The 3D extension on one point set of n points (n in [0, 2^32 - 1]).
 *   d_survivor_idx   room for n uint32: the points not strictly inside the
 *                    polyhedron, in unspecified order (compare as a set).
 *   d_n_survivors    one int64: their number.
 *   d_extreme_idx    24 uint32 (may be NULL): the extremes, see above; all
 *                    0xFFFFFFFF when n == 0.
 * The polyhedron stays in the workspace (hull3_read_polyhedron). */
hull_status hull3_prefilter(const float* d_xyz, int64_t n, void* d_ws, size_t ws_bytes, uint32_t* d_survivor_idx,
                            int64_t* d_n_survivors, uint32_t* d_extreme_idx, const hull_options* opt, void* stream);

/* The polyhedron of the last hull3_prefilter on this workspace (host
 * memory; synchronises the stream): *h_nf facets, h_planes[4k .. 4k+3] =
 * Nx, Ny, Nz, d of facet k (room for 4 * HULL3_MAX_FACETS int64; may be
 * NULL), h_ext the 24 extremes (may be NULL), h_counts[3] = survivors,
 * float32 plane tests escalated to int64, device status bits (may be NULL). */
hull_status hull3_read_polyhedron(const void* d_ws, int32_t* h_nf, int64_t* h_planes, uint32_t* h_ext,
                                  int64_t* h_counts, void* stream);

/* ---- Instrumentation (not part of the method) -------------------------- */

/* Stages of one call, in launch order: domain check (and batch set-up),
 * the streaming extreme search (Step 1), the polygon of the extremes and
 * its cell grid (Step 2), inside test + compaction (Step 3), the
 * refinement round and the small-set hull, the large-set hull. */
#define HULL_STAGES 6

/* Opaque stage timer: CUDA events recorded on the call's stream at every
 * stage boundary (host objects; no device memory). */
typedef struct hull_timer hull_timer;

/* Creates a timer with room for max_calls calls; NULL on failure. */
hull_timer* hull_timer_create(int32_t max_calls);
void hull_timer_destroy(hull_timer* t);

/* Subsequent hull_prefilter / hull_compute calls made by this host thread
 * record their stage boundaries into t (NULL detaches).  Calls beyond the
 * timer's capacity are not recorded. */
void hull_timer_attach(hull_timer* t);

/* Waits for the recorded events, writes the per-stage time summed over the
 * recorded calls to h_ms[HULL_STAGES] (milliseconds) and the number of
 * recorded calls to *h_calls, then clears the timer. */
hull_status hull_timer_read(hull_timer* t, float* h_ms, int32_t* h_calls);

/* Number of kernels this library has enqueued in this process so far. */
int64_t hull_launch_count(void);

/* Test of the timeout path (no counterpart in the paper): one kernel waits,
 * with a limit of limit_cycles GPU cycles (1 .. 2^31), on a barrier that
 * nothing releases; the wait gives up, records HULL_DEVICE_TIMEOUT in d_ws's
 * status word (cleared first) and the kernel returns.  The context stays
 * usable; hull_get_device_status then reports HULL_ERR_TIMEOUT.  d_ws: any
 * workspace (256-byte aligned). */
hull_status hull_selftest_wait(void* d_ws, int64_t limit_cycles, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CUDAPRE_H */
