/*
 * fastatlas.h - C ABI of the GB300 (sm_103a) per-frame atlasing path of
 * FastAtlas (Vining et al., "FastAtlas: Real-Time Compact Atlases for Texture
 * Space Shading", EG 2025).
 *
 * One frame: find the visible triangles (Sec. 5.1, App. A), group them into
 * charts (connected components, Sec. 5.1, Alg. 1), give each chart a
 * conservative projected box and quantized footprint (Sec. 5.2, Sec. 4.1), pack
 * the footprints into an omega x omega atlas by the 64-scale prefix-sum fold /
 * push search (Sec. 4.2, 4.3), and map every visible corner into its chart's
 * atlas box (Sec. 3, App. A "Shading and Rasterization").
 *
 * Conventions shared by every call:
 *  - Pointers named d_* are DEVICE pointers owned by the caller; host pointers
 *    are read before the call returns.  The library never frees caller memory.
 *  - Scratch memory is owned by the context and allocated once in fa_create
 *    for the configured maxima; no per-frame call allocates, synchronizes or
 *    copies to the host, so the calls may be captured in a CUDA graph.
 *  - Every call is asynchronous and stream ordered on `stream` (a cudaStream_t;
 *    NULL is the legacy default stream).  Argument errors the host can see are
 *    returned immediately and nothing is launched.  Errors found on the device
 *    (too many charts, no fitting scale, an iteration cap hit) are written to the
 *    context's sticky device status word and, for packing, to
 *    fa_pack_result.status; later kernels of the same context see the word and
 *    skip their work.  fa_last_device_status reads and clears it.
 *  - A context is not thread safe: use one context per stream / session.
 *  - Matrices are row major float[16]; clip = M . [x, y, z, 1].  OpenGL
 *    conventions: the near plane is z_clip = -w_clip, screen y points up, front
 *    faces are counter-clockwise on screen.
 */
#ifndef FASTATLAS_H_
#define FASTATLAS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* fa_stream_t; /* same type as cudaStream_t */

typedef enum {
  FA_OK = 0,
  FA_E_INVALID_ARG = 1,   /* bad pointer, size or parameter; nothing launched   */
  FA_E_OUT_OF_MEMORY = 2, /* fa_create / fa_mesh_register could not allocate      */
  FA_E_CAPACITY = 3,      /* a configured maximum was exceeded (charts, frontline) */
  FA_E_PACK_FAILED = 4,   /* no candidate scale fits the atlas (Sec. 4.2)          */
  FA_E_TIMEOUT = 5,       /* a device loop hit its iteration cap                   */
  FA_E_CUDA = 6           /* a CUDA runtime call failed                           */
} fa_status;

typedef enum {
  FA_CHARTS_EDGE = 0,   /* components under shared edges (Sec. 5.1)                  */
  FA_CHARTS_VERTEX = 1  /* components under shared vertices: the vertex merge that
                           gives every vertex one chart (App. A, Alg. 1)              */
} fa_chart_mode;

typedef enum {
  FA_SELECT_EFFECTIVE = 0, /* largest effective scale (k/n) * omega / Omega        */
  FA_SELECT_LARGEST_K = 1  /* largest fitting candidate k (Sec. 4.2 literal)         */
} fa_select_mode;

/* Context maxima.  Scratch is sized from these once, in fa_create. */
typedef struct {
  uint32_t max_tris;       /* triangles of the largest registered mesh              */
  uint32_t max_verts;      /* vertices of the largest registered mesh               */
  uint32_t max_charts;     /* charts per frame (paper: "user-defined maximal number
                              of charts", data structures table); at most 1<<22     */
  uint32_t max_width;      /* largest viewport, pixels (<= 16384)                   */
  uint32_t max_height;
  uint32_t max_atlas_log2; /* largest atlas side omega = 2^log2 (<= 14)             */
  uint32_t min_box;        /* smallest packed box side in texels (paper: 2)        */
  uint32_t gutter;         /* texels added on every side of a packed box (0)       */
  int32_t device;          /* CUDA device ordinal                                   */
} fa_config;

typedef struct fa_ctx fa_ctx;
typedef struct fa_mesh fa_mesh;

/* Per-chart arrays (structure of arrays, caller-owned device memory, each with
 * room for fa_config.max_charts entries). */
typedef struct {
  uint32_t* root;  /* smallest triangle id of the chart; charts numbered by root   */
  float* bbox;     /* [C][4] xmin, ymin, xmax, ymax of the conservative NDC box    */
  uint32_t* fa;    /* [C] footprint width in 1/256 texel after rotation (fa <= fb) */
  uint32_t* fb;    /* [C] footprint height in 1/256 texel                          */
  uint8_t* rot;    /* [C] 1 if the box was rotated by 90 degrees to stand tall     */
  uint32_t* count; /* [1] number of charts C of the frame                          */
} fa_charts;

/* Placement of one chart in the chosen candidate's virtual Omega x Omega grid; the
 * real atlas rectangle is alpha * [x, x + w) x alpha * [y, y + h), alpha = omega /
 * Omega, and the chart's content starts gutter texels inside it. */
typedef struct {
  int32_t x, y, w, h;
} fa_placement;

typedef struct {
  uint32_t k;      /* chosen scale numerator: scale = k / n_scales                 */
  uint32_t omega;  /* virtual side Omega = omega + m of the chosen candidate       */
  uint32_t height; /* stacked height H <= Omega                                    */
  int32_t status;  /* fa_status of the packing                                     */
  uint32_t count;  /* number of boxes packed                                       */
} fa_pack_result;

typedef struct {
  float view_proj[16];  /* row major, clip = M . [p, 1]                            */
  uint32_t width;       /* viewport, pixels                                        */
  uint32_t height;
  float ratio;          /* texel-to-pixel ratio r (linear, per axis; 0 < r <= 64) */
  uint32_t atlas_log2;  /* omega = 2^atlas_log2                                    */
  uint32_t chart_mode;  /* fa_chart_mode                                           */
  uint32_t n_scales;    /* candidate scales k / n, k = 1..n; n in {1,2,4,...,64}   */
  uint32_t select_mode; /* fa_select_mode                                          */
  uint32_t flags;       /* FA_BOX_FRUSTUM_CLIP | FA_VIS_CONSERVATIVE | FA_LOWRES(d) |
                           FA_FRAME_PERSISTENT */
} fa_frame_params;

/* fa_frame_params.flags / fa_parameterize flags.  FA_BOX_FRUSTUM_CLIP: a visible
 * triangle that does not cross the near plane is clipped against the one frustum
 * plane (left, right, bottom, top, far, in this order) whose single-plane clip
 * gives the smallest Blinn box, fp32 area (xmax - xmin) * (ymax - ymin), ties to
 * the earlier plane, before Blinn's clamp (Sec. 5.2: the second clip whose details
 * the paper leaves to its supplementary material).  Tighter, still conservative. */
#define FA_BOX_FRUSTUM_CLIP 1u

/* fa_frame_params.flags / fa_visibility flags.  FA_VIS_CONSERVATIVE: the marking
 * pass rasterizes conservatively, as the paper's does (App. A): a pixel counts
 * when its closed square meets the closed (snapped, culled) sub-triangle, with the
 * pre-pass depth where the sample rule covers its centre and otherwise the plane
 * extrapolated to the centre and clamped to the sub-triangle's vertex depths; the
 * triangle is visible when such a pixel passes the "<=" test.  The depth pre-pass
 * keeps the sample rule.  Marks a superset of the default's triangles. */
#define FA_VIS_CONSERVATIVE 2u

/* fa_frame_params.flags bits 8..10: one packing, two atlases (Sec. 7: depth of
 * field and foveated rendering shade a second atlas of the same packing scaled by
 * 2^-d).  With d > 0 a candidate is accepted only if also
 * 2 * gutter * omega >= Omega * 2^d: the contents of two charts, at least
 * 2 * gutter virtual texels (2 * gutter * omega / Omega atlas texels) apart, then
 * share no texel of the scaled atlas.  Needs a context gutter > 0.  The scaled
 * atlas's UVs are the UVs times 2^-d (exact in fp32). */
#define FA_LOWRES(d) ((((uint32_t)(d)) & 7u) << 8)

/* fa_frame_params.flags: run the whole frame as ONE launch of the persistent frame
 * kernel instead of the 15-launch sequence.  A cooperative grid of one CTA per SM
 * takes (stage, worker) items in order from a device queue; a stage starts when the
 * stage before it has finished (a device counter instead of a kernel boundary).
 * The stages run the same code as the separate kernels, so the results are
 * identical; on small frames the launch and drain of every kernel of the sequence
 * dominate, and this removes them.  Works with every other flag, chart mode and
 * output, in fa_atlas_frame, fa_atlas_frame_dev_matrix, batches and the server. */
#define FA_FRAME_PERSISTENT (1u << 12)

/* All outputs of fa_atlas_frame (caller-owned device memory). */
typedef struct {
  uint32_t* vt;           /* [ceil(T/32)] visible-triangle bits                     */
  int32_t* tri_chart;     /* [T] chart of each triangle, -1 if not visible          */
  int32_t* vert_chart;    /* [V] chart of each vertex (vertex mode), -1 if none; may
                             be NULL                                                */
  fa_charts charts;       /* per-chart arrays                                       */
  uint32_t* order;        /* [max_charts] packing order; may be NULL                */
  fa_placement* place;    /* [max_charts] placements, chart order                   */
  fa_pack_result* result; /* [1]                                                    */
  float* uv;              /* [T][3][2] atlas texel coordinates per visible corner;
                             NaN where w <= 0; untouched for invisible triangles; may
                             be NULL                                                */
  float* affine;          /* [max_charts][6] (a11, a12, b1, a21, a22, b2):
                             uv = A . ndc + b, i.e. uv * w = A . (x, y) + b * w;
                             may be NULL                                            */
  uint32_t* partial;      /* [ceil(T/32)] partially visible triangles (visible, with a
                             vertex where max(|x|, |y|) >= w in clip coordinates;
                             Sec. 6 temporal re-use shades these again); may be NULL */
} fa_frame_out;

/* Library version (major * 10000 + minor * 100 + patch). */
uint32_t fa_version(void);

/* Human readable name of a status code (static storage). */
const char* fa_status_string(fa_status s);

/* Create a context on cfg->device and allocate its scratch for the maxima in cfg
 * (once; the paper likewise allocates its scratch "at the start of program
 * execution", Sec. 4.1).  *out is set to NULL on failure.
 * Errors: FA_E_INVALID_ARG (NULL pointers, zero or too large maxima),
 * FA_E_OUT_OF_MEMORY, FA_E_CUDA. */
fa_status fa_create(fa_ctx** out, const fa_config* cfg);

/* Free the context and its scratch.  Waits for the device.  NULL is ignored. */
void fa_destroy(fa_ctx* ctx);

/* Register a triangle mesh: d_pos float[V][3] positions, d_idx uint32[T][3]
 * CCW index triples (both caller-owned, kept by pointer: positions may be
 * rewritten between frames, the topology may not).  Builds the triangle
 * adjacency that Alg. 1 walks (the half-edge twins of the data-structures
 * table) once on the device: two triangles are adjacent when they share an
 * undirected edge {a, b}, a != b, of the index buffer; an edge with three or more
 * triangles (non-manifold) joins all of them.  This call allocates the mesh's own
 * device buffers and synchronizes `stream`; it is set-up, not per-frame work.
 * Errors: FA_E_INVALID_ARG (T > max_tris, V > max_verts, an index >= V is
 * reported as FA_E_INVALID_ARG after the synchronizing check), FA_E_OUT_OF_MEMORY,
 * FA_E_CUDA. */
fa_status fa_mesh_register(fa_ctx* ctx, const float* d_pos, uint32_t V, const uint32_t* d_idx,
                           uint32_t T, fa_mesh** out, fa_stream_t stream);

/* Free a mesh's device buffers (waits for the device).  NULL is ignored. */
void fa_mesh_release(fa_mesh* mesh);

/* Visible triangles (Sec. 5.1; App. A "Detecting Visible Triangles"): a depth
 * pre-pass over the width x height viewport, then a marking pass in which a
 * triangle is visible iff one of its samples passes the "less than or equal"
 * depth test.  Samples are pixel centres; coverage uses the top-left rule on
 * vertices snapped to 1/256 pixel after clipping against the near plane and a
 * guard band |x|, |y| <= 64 w; back faces and zero-area triangles are culled.
 * flags: 0, or FA_VIS_CONSERVATIVE for the conservative marking pass.
 * d_vt: uint32[ceil(T/32)], bit t%32 of word t/32 (fully overwritten).
 * Errors: FA_E_INVALID_ARG (viewport above the context maximum, NULL pointers,
 * unknown flags). */
fa_status fa_visibility(fa_ctx* ctx, const fa_mesh* mesh, const float view_proj[16],
                        uint32_t width, uint32_t height, uint32_t flags, uint32_t* d_vt,
                        fa_stream_t stream);

/* Charts (Sec. 5.1; App. A "GPU Union Find", Alg. 1): connected components of
 * the visible triangles under shared edges (FA_CHARTS_EDGE) or shared vertices
 * (FA_CHARTS_VERTEX).  A chart's root is its smallest triangle id, and charts are
 * numbered by ascending root.  Writes d_tri_chart int32[T] (-1 = invisible),
 * charts->root and charts->count; d_vert_chart int32[V] (may be NULL) gets each
 * vertex's chart in vertex mode and -1 otherwise.  More than max_charts charts
 * sets FA_E_CAPACITY in the device status word (outputs then undefined).
 * Errors: FA_E_INVALID_ARG. */
fa_status fa_chartify(fa_ctx* ctx, const fa_mesh* mesh, const uint32_t* d_vt, uint32_t mode,
                      int32_t* d_tri_chart, int32_t* d_vert_chart, const fa_charts* charts,
                      fa_stream_t stream);

/* Chart boxes and footprints (Sec. 5.2, Sec. 4.1): each visible triangle is
 * clipped against the near plane when it crosses it, each remaining vertex is
 * clamped to [-w, w] and divided (Blinn's estimator), and the chart box is the
 * min / max over its triangles (a vertex with w <= 0 left after the near clip
 * makes the box [-1,1]^2).  The box's viewport size is scaled by `ratio`,
 * quantized up to 1/256 texel, and rotated to stand tall (fa <= fb, rot = 1 when
 * the width exceeded the height).  Reads charts->count; writes bbox, fa, fb, rot.
 * flags: FA_BOX_FRUSTUM_CLIP or 0.  d_partial (may be NULL): [ceil(T/32)] bits of
 * the partially visible triangles (see fa_frame_out.partial), cleared first.
 * Errors: FA_E_INVALID_ARG. */
fa_status fa_parameterize(fa_ctx* ctx, const fa_mesh* mesh, const float view_proj[16],
                          uint32_t width, uint32_t height, float ratio,
                          const int32_t* d_tri_chart, const fa_charts* charts, uint32_t flags,
                          uint32_t* d_partial, fa_stream_t stream);

/* Packing (Sec. 4.1-4.3).  Inputs: d_count[0] boxes with footprints d_fa, d_fb in
 * 1/256 texel (the box index is the tie-break of the order, so pass boxes by
 * ascending root for the paper's order).  Order: integer height ceil(fb/256)
 * (clamped to [1, 8192]) descending, index ascending.  Candidates k = 1..n_scales
 * (n_scales a power of two <= 64): box w = max(min_box, ceil(k fa / (256 n))) +
 * 2 gutter (same for h from fb); the exclusive prefix sum P of the widths gives
 * row = P >> atlas_log2 and offset P & (omega - 1); m = the largest overflow past
 * omega, Omega = omega + m; rows with row % 3 == 0 run left to right, the others
 * right to left mirrored in Omega; rows are then pushed up against the frontline.
 * A candidate fits iff its height H <= Omega.  The selected candidate is written
 * to *d_res and its placements (chart order) to d_place; d_order (may be NULL)
 * receives the packing order.  No fitting candidate: d_res->status =
 * FA_E_PACK_FAILED.  A candidate with Omega above the frontline capacity
 * min(8 omega, 32768) sets FA_E_CAPACITY.  lowres_log2 = d > 0: candidates must
 * also serve the atlas scaled by 2^-d (see FA_LOWRES); 0 for none.
 * Errors: FA_E_INVALID_ARG (atlas_log2 out of range, n_scales not a power of two
 * in [1, 64], select_mode unknown, lowres_log2 > 7, NULL pointers). */
fa_status fa_pack(fa_ctx* ctx, const uint32_t* d_fa, const uint32_t* d_fb, const uint32_t* d_count,
                  uint32_t atlas_log2, uint32_t n_scales, uint32_t select_mode, uint32_t* d_order,
                  fa_placement* d_place, fa_pack_result* d_res, uint32_t lowres_log2, fa_stream_t stream);

/* Packing without any allocation.  The paper has no counterpart: this is a
 * service for callers that may not allocate device memory where they pack, such as
 * code running in a host application's per-frame callback or plugin slot whose
 * device memory is owned and budgeted by the host, or a real-time loop that must
 * not pay cudaMalloc's implicit device synchronization.  It computes exactly what
 * fa_pack computes (same order, candidates, selection and placements) for n boxes
 * d_fa, d_fb (n given on the host), with min_box and gutter passed directly, and
 * needs no context.
 * Scratch: one file-scope device array of about 4.8 MiB inside the library, sized
 * for at most 4096 boxes; every GPU that loads the library holds it until the
 * process exits.  The call never runs cudaMalloc, cudaFree or any allocating
 * library routine.
 * The first call on a device looks up the array's device address (with that device
 * current) and raises the pack kernel's shared-memory limit; make that first call
 * before any stream capture.  Later calls only launch kernels on `stream`, on the
 * current device.  The address is kept for the life of the process: resetting the
 * device (cudaDeviceReset, or tearing down its primary context) afterwards is not
 * supported.
 * All calls share the one array, and each call leaves its contents behind (the
 * call clears what must start at zero itself); calls whose kernels overlap on the
 * GPU (different streams, or different host threads) race on it and must be
 * serialized by the caller.
 * Errors: FA_E_CAPACITY (n > 4096), FA_E_INVALID_ARG (NULL pointers, atlas_log2
 * outside [1, 14], n_scales not a power of two in [1, 64], unknown select_mode,
 * min_box outside [1, 4096], gutter > 4096), FA_E_CUDA (set-up or launch failed);
 * device-side results and errors land in d_res as for fa_pack. */
fa_status fa_pack_noalloc(const uint32_t* d_fa, const uint32_t* d_fb, uint32_t n, uint32_t atlas_log2,
                          uint32_t n_scales, uint32_t select_mode, uint32_t min_box, uint32_t gutter,
                          uint32_t* d_order, fa_placement* d_place, fa_pack_result* d_res,
                          fa_stream_t stream);

/* Parameterization (Sec. 3; App. A "Shading and Rasterization"): every visible
 * corner with w > 0 maps to alpha * ((x + gutter, y + gutter) + s * local) in atlas
 * texels, alpha = omega / Omega, s = ratio * k / n_scales, local = the corner's
 * viewport position relative to the chart box, rotated by +90 degrees for rotated
 * charts (local = (py, Wpx - px)).  Computed from the fp32 clip coordinates with
 * compensated fp32 arithmetic and rounded once: within 1e-4 texel of the exact
 * value wherever fp32 can hold it to 1e-4 (|uv| < 2048, every corner inside an
 * atlas of side <= 2048), else the correctly rounded fp32 value (half an ulp,
 * plus 2^-30 |uv|).  d_uv float[T][3][2] (NaN for w <= 0,
 * untouched for invisible triangles), d_affine float[C][6] (may be NULL).
 * Skipped when d_res->status != FA_OK.  Errors: FA_E_INVALID_ARG. */
fa_status fa_uv(fa_ctx* ctx, const fa_mesh* mesh, const float view_proj[16], uint32_t width,
                uint32_t height, float ratio, const int32_t* d_tri_chart, const fa_charts* charts,
                const fa_placement* d_place, const fa_pack_result* d_res, uint32_t atlas_log2,
                uint32_t n_scales, float* d_uv, float* d_affine, fa_stream_t stream);

/* The whole per-frame path: fa_visibility, fa_chartify, fa_parameterize,
 * fa_pack and fa_uv in one stream-ordered launch sequence (device status word
 * cleared first).  Errors: FA_E_INVALID_ARG (as for the steps). */
fa_status fa_atlas_frame(fa_ctx* ctx, const fa_mesh* mesh, const fa_frame_params* params,
                         const fa_frame_out* out, fa_stream_t stream);

/* fa_atlas_frame with the view-projection matrix read on the device, when the
 * kernels run, from d_view_proj (16 floats, row-major as in params->view_proj,
 * 16-byte aligned, caller-owned); params->view_proj is ignored.  The paper
 * re-atlases every frame along a camera path (Sec. 6, per-frame timings over
 * camera paths): a CUDA graph captured from one call of this function serves the
 * whole path, the caller writing the next camera into d_view_proj (stream-ordered)
 * before each replay.  Results equal fa_atlas_frame's for the same matrix.
 * Errors: FA_E_INVALID_ARG (as fa_atlas_frame, or d_view_proj NULL / misaligned). */
fa_status fa_atlas_frame_dev_matrix(fa_ctx* ctx, const fa_mesh* mesh, const fa_frame_params* params,
                                    const float* d_view_proj, const fa_frame_out* out, fa_stream_t stream);

/* Synchronize `stream`, read the context's sticky device status word into *out
 * and clear it.  Returns FA_E_CUDA if the stream reported a CUDA error. */
fa_status fa_last_device_status(fa_ctx* ctx, fa_stream_t stream, int32_t* out);

/* Limits of the device-side waits in this context's later launches.  The paper
 * has no failure detection; these bound every loop of the library that waits on
 * other threads, so that a fault elsewhere cannot hang the GPU.
 *  loop_cap: CAS retries of one union-find hooking step (Alg. 1's hooking loop);
 *            also caps the polls (at most 256) of the packing width scan's
 *            look-back on an earlier chunk that has published nothing, after which
 *            the scan sums that chunk's widths itself (it never runs out);
 *  wait_ns:  nanoseconds the packing push waits for a chunk's bulk copy.
 * When a limit runs out the kernel writes FA_E_TIMEOUT to the device status word,
 * drops its remaining work (later kernels of the call see the word and skip
 * theirs; fa_pack_result.status reports it) and returns; copies it started are
 * still waited for, up to FA_DEFAULT_WAIT_NS, before it exits.  The context stays
 * usable: the next frame starts from a cleared status word.  The defaults lie far
 * above what any frame needs; small values exist to exercise the time-out path.
 * Kernels launched after the call use the new limits (a CUDA graph keeps those of
 * its capture).  Errors: FA_E_INVALID_ARG (NULL ctx). */
#define FA_DEFAULT_LOOP_CAP (1u << 24)
#define FA_DEFAULT_WAIT_NS 1000000000ull
fa_status fa_set_wait_limits(fa_ctx* ctx, uint32_t loop_cap, uint64_t wait_ns);

/* Raster schedule of this context's later frames (changes timing only, never
 * results).
 *  mid_max_pix: a sub-triangle whose pixel box has at most 16 pixels is rasterized
 *    by one thread; larger ones are split into 16x16 tiles, one warp per tile.
 *    With mid_max_pix > 16, boxes of up to mid_max_pix pixels are also rasterized
 *    in-thread when, for the warp that set them up, that costs less than the tiles
 *    (the warp's largest such box against the summed tile steps).  That pays on
 *    views of many mid-size triangles (high resolutions, dense meshes seen close
 *    up); on views of mostly tiny triangles the tiles stay cheaper, hence the
 *    default FA_RASTER_MID_OFF.
 *  flags: FA_RASTER_HIZ adds a pass that takes the largest depth of every 16x16
 *    pixel tile of the final depth buffer; the marking pass then skips a
 *    sub-triangle (or a tile of one) whose smallest possible sample depth, less a
 *    bound on the depth's rounding error, is above the largest depth of every tile
 *    it touches.  That pays where most hidden triangles lie behind fully covered
 *    tiles (large overlapping surfaces); off by default.
 * Both ways the same samples get the same depth keys and the same triangles are
 * marked.  Errors: FA_E_INVALID_ARG (NULL ctx, mid_max_pix outside [16, 256],
 * unknown flags). */
#define FA_RASTER_MID_OFF 16u
#define FA_RASTER_MID_MAX 256u
#define FA_RASTER_HIZ 1u
fa_status fa_set_raster_schedule(fa_ctx* ctx, uint32_t mid_max_pix, uint32_t flags);

/* Kernel shapes of the chart and packing passes on this context, a schedule knob
 * like the raster one: every value gives the same results, only the timing differs.
 *   uf_threads    threads per 1024-triangle tile of the local union-find of the chart
 *                 pass (App. A "GPU Union Find"): 256, 512 or 1024 (4, 2 or 1
 *                 triangles per thread; 8, 4 or 2 tiles resident per SM);
 *   push_threads  threads of the CTA that pushes one scale candidate's rows onto its
 *                 frontline (Sec. 4.3): 256, 512 or 1024.
 * Defaults 1024 and 512 (the fastest on one large frame).  fa_batch_tune searches both.
 * The persistent frame kernel (FA_FRAME_PERSISTENT, batch plans) runs its own
 * 1024-thread CTAs and ignores them.
 * Errors: FA_E_INVALID_ARG (NULL ctx, any other value). */
fa_status fa_set_chart_pack_schedule(fa_ctx* ctx, uint32_t uf_threads, uint32_t push_threads);

/* The schedule knobs of a context (fa_set_raster_schedule, fa_set_chart_pack_schedule).
 * Errors: FA_E_INVALID_ARG (NULL ctx or out). */
typedef struct fa_kernel_schedule {
  uint32_t mid_max_pix;
  uint32_t raster_flags;
  uint32_t uf_threads;
  uint32_t push_threads;
} fa_kernel_schedule;
fa_status fa_get_kernel_schedule(const fa_ctx* ctx, fa_kernel_schedule* out);

/* Number of kernels the library launched on this context since creation (a
 * host-side counter; used to report launches per frame). */
uint64_t fa_launch_count(const fa_ctx* ctx);

/* Work counts of the last frame (or fa_visibility / fa_chartify call) on this
 * context, read from its device counters after synchronizing `stream`.  They
 * describe how much work the data-dependent kernels had (the benchmark derives
 * their compulsory bytes from them) and change no result.
 * Errors: FA_E_INVALID_ARG (NULL ctx or out), FA_E_CUDA. */
typedef struct fa_frame_stats {
  uint32_t survivors;     /* triangles that passed the raster front end */
  uint32_t clipped;       /* of those, triangles that needed clipping */
  uint32_t clip_records;  /* small sub-triangle records of the clipping path */
  uint32_t big_entries;   /* large sub-triangles queued for tile rasterization */
  uint64_t big_tiles;     /* their 16x16 tiles */
  uint32_t visible;       /* entries of the visible-triangle list */
  uint32_t charts;        /* charts of the last chart pass */
  uint32_t visible_tiles; /* tiles of 1024 consecutive triangles holding a visible one */
} fa_frame_stats;
fa_status fa_frame_stats_read(fa_ctx* ctx, fa_stream_t stream, fa_frame_stats* out);

/* Per-kernel tracing (the paper times its stages per frame, App. B "Timing
 * Methodology"; here every kernel of a public call gets a slot).  When enabled,
 * each public call records a CUDA event on `stream` before each of its kernels
 * and one after the last, so slot i spans kernel i (and any launch gap before
 * kernel i + 1).  Recording works inside CUDA-graph capture: a replay then
 * re-records the same events.  fa_profile_enable(ctx, 1) creates the events (call
 * it outside any capture); 0 destroys them.  Errors: FA_E_INVALID_ARG, FA_E_CUDA. */
fa_status fa_profile_enable(fa_ctx* ctx, int enable);

/* Wait for the last traced call to finish and return up to max_n slot durations
 * in milliseconds (ms[i]) with the kernel names (names[i], static strings); *n_out
 * receives the number of slots of that call (0 when tracing is off).
 * Errors: FA_E_INVALID_ARG, FA_E_CUDA. */
fa_status fa_profile_read(fa_ctx* ctx, int max_n, float* ms, const char** names, int* n_out);

/* ------------------------------------------------------------------ batches
 *
 * Many independent views atlased together.  Each view is one frame of the path
 * above (its own mesh, camera, viewport, ratio and atlas; Sec. 3: one atlas per
 * view); a batch runs them on lanes, each lane a context with its own stream,
 * forked from and joined back into the caller's stream.  Results equal
 * fa_atlas_frame's for every view, whatever the schedule.  A CUDA graph captured
 * from one fa_atlas_batch call atlases the whole batch in one launch. */
typedef struct fa_batch fa_batch;

typedef enum {
  FA_BATCH_ROUND_ROBIN = 0,   /* view i on lane i mod lanes */
  FA_BATCH_LONGEST_FIRST = 1  /* views by decreasing T + W*H, each to the least-loaded lane */
} fa_batch_policy;

#define FA_BATCH_MAX_LANES 64u

/* n_lanes contexts of configuration *cfg (device memory: n_lanes times one
 * context) and their streams; all lanes in use, round robin.
 * Errors: FA_E_INVALID_ARG (n_lanes 0 or above FA_BATCH_MAX_LANES, bad cfg),
 * FA_E_OUT_OF_MEMORY, FA_E_CUDA. */
fa_status fa_batch_create(fa_batch** out, const fa_config* cfg, uint32_t n_lanes);

/* Synchronizes the device and frees the lanes.  Release the batch's meshes first. */
void fa_batch_destroy(fa_batch* batch);

/* fa_mesh_register for a mesh used in this batch's views (any lane may run it). */
fa_status fa_batch_mesh_register(fa_batch* batch, const float* d_pos, uint32_t V, const uint32_t* d_idx,
                                 uint32_t T, fa_mesh** out, fa_stream_t stream);

/* Lanes in use (1 .. n_lanes) and the assignment policy of later calls. */
fa_status fa_batch_set_schedule(fa_batch* batch, uint32_t lanes, uint32_t policy);
fa_status fa_batch_get_schedule(const fa_batch* batch, uint32_t* lanes, uint32_t* policy);

/* Enqueue n_views frames: view i = meshes[i] (registered with this batch) with
 * params[i] into outs[i] (caller-owned, distinct per view).  Every view is checked
 * on the host before anything is enqueued.  Each view's own result status is in
 * outs[i].result.  Errors: FA_E_INVALID_ARG, FA_E_CUDA. */
fa_status fa_atlas_batch(fa_batch* batch, uint32_t n_views, const fa_mesh* const* meshes,
                         const fa_frame_params* params, const fa_frame_out* outs, fa_stream_t stream);

/* Schedule autotuner: first the raster schedule of every lane's context (mid-size
 * limit 16 or 64, with and without FA_RASTER_HIZ, at the current lanes), then the
 * chart/pack kernel shapes (uf_threads x push_threads in {256, 512, 1024}^2), then
 * lanes in {1, 2, 4, .., n_lanes} x both policies: each schedule's batch is captured into
 * a CUDA graph, launched once, `reps` launches are timed (CUDA events, best of) and
 * the fastest schedule is kept; *best_ms (may be NULL)
 * receives its time.  Runs the views (outputs are overwritten) and synchronizes;
 * not for use inside a capture.  Errors: FA_E_INVALID_ARG, FA_E_CUDA. */
fa_status fa_batch_tune(fa_batch* batch, uint32_t n_views, const fa_mesh* const* meshes,
                        const fa_frame_params* params, const fa_frame_out* outs, uint32_t reps,
                        float* best_ms);

/* The kernel schedule of the batch's lanes (all lanes share it; the tuner sets it). */
fa_status fa_batch_get_kernel_schedule(const fa_batch* batch, fa_kernel_schedule* out);

/* Kernels launched by all lanes since creation. */
uint64_t fa_batch_launch_count(const fa_batch* batch);

/* Batch plans: the views of a batch atlased by ONE launch of the persistent frame
 * kernel (see FA_FRAME_PERSISTENT).  The launch is a cooperative grid of one
 * 1024-thread CTA per SM that drains a device work queue of (view, stage, worker)
 * items: a stage is one step of the per-frame path (raster front end, exact
 * set-up, large-triangle tiles, marking, the union-find passes, chart ids, boxes,
 * order, width scan, push, UVs), its workers are the virtual blocks of that step's
 * kernel.  Items are claimed in a fixed order: round by round (the r-th view of
 * every lane), stage by stage, lane by lane; an item waits until the stage before
 * it has finished (and a view's first stage until the lane's previous view has).
 * While one view's latency-bound stages leave SMs idle, the other views' stages run
 * there.  Results equal fa_atlas_frame's for every view.  A plan is set-up work:
 * creating or rescheduling it builds and uploads the views' arguments and
 * synchronizes the device; launching it only enqueues the one kernel, so a CUDA
 * graph captured from fa_batch_plan_launch atlases the batch in one kernel node.
 * The views' matrices are params[i].view_proj, or read on the device when the
 * kernel runs from d_view_proj[i] (16 floats, 16-byte aligned) when d_view_proj is
 * given, so a captured launch can serve new cameras.  Meshes, outputs and matrix
 * buffers must stay alive and in place while the plan is used. */
typedef struct fa_batch_plan fa_batch_plan;

#define FA_PLAN_MAX_VIEWS 4096u

/* Schedule of a plan; it changes timing only, never results. */
typedef struct {
  uint32_t lanes;       /* lanes (contexts) used, 1 .. the batch's n_lanes; a lane's views run in turn */
  uint32_t policy;      /* fa_batch_policy: views to lanes */
  uint32_t worker_pct;  /* workers per data-sized stage, percent of the default counts (10 .. 1000) */
  uint32_t mid_max_pix; /* raster schedule of every view (see fa_set_raster_schedule) */
  uint32_t raster_flags;
} fa_plan_schedule;

/* Plan n_views views (as fa_atlas_batch) on all of the batch's lanes, longest
 * first, default worker counts.  d_view_proj may be NULL.
 * Errors: FA_E_INVALID_ARG (a view fails fa_atlas_frame's checks, n_views 0 or above
 * FA_PLAN_MAX_VIEWS), FA_E_OUT_OF_MEMORY, FA_E_CUDA. */
fa_status fa_batch_plan_create(fa_batch* batch, uint32_t n_views, const fa_mesh* const* meshes,
                               const fa_frame_params* params, const float* const* d_view_proj,
                               const fa_frame_out* outs, fa_batch_plan** out);

/* One launch of the persistent kernel for every view of the plan on `stream`.  Each
 * view's status lands in its result record (FA_E_TIMEOUT for every view if a wait
 * of the launch ran out).  Launches of one plan must not overlap on the GPU.
 * Errors: FA_E_INVALID_ARG, FA_E_CUDA. */
fa_status fa_batch_plan_launch(fa_batch_plan* plan, fa_stream_t stream);

/* Read / change the schedule (changing it rebuilds the plan; synchronizes). */
fa_status fa_batch_plan_get_schedule(const fa_batch_plan* plan, fa_plan_schedule* schedule);
fa_status fa_batch_plan_set_schedule(fa_batch_plan* plan, const fa_plan_schedule* schedule);

/* Schedule autotuner: lanes in {1, 2, 4, .., n_lanes} x both policies x worker
 * counts at 50 / 100 / 200 %, after the raster schedule (mid-size limit 16 or 64,
 * with and without FA_RASTER_HIZ) was picked on all lanes; each schedule is
 * launched once, then `reps` launches are timed (CUDA events, best of); the
 * fastest is kept.  Runs the views (outputs
 * are overwritten) and synchronizes; not for use inside a capture.  *best_ms (may
 * be NULL) receives its time.  Errors: FA_E_INVALID_ARG, FA_E_CUDA. */
fa_status fa_batch_plan_tune(fa_batch_plan* plan, uint32_t reps, float* best_ms);

/* Synchronizes the device and frees the plan.  NULL is ignored. */
void fa_batch_plan_destroy(fa_batch_plan* plan);

/* ------------------------------------------------------------------ serving
 *
 * Continuous batching of per-client view requests.  The paper's setting is a
 * streaming-shading server that re-atlases every client frame (Sec. 1, Sec. 6);
 * here clients are sessions whose mesh and output buffers stay on the device.
 * The server owns slots (a context plus a stream each), as many as fit a
 * device-memory budget.  Requests are queued when submitted and dispatched, in
 * submission order, to the first free slot once their session has no request on
 * the GPU; a request that arrives while others run starts as soon as a slot frees
 * up, and the slots' work overlaps on the device.  Each request runs the
 * fa_atlas_frame launch sequence, so its results equal those of the same request
 * alone.  The server is driven from one host thread (submit / poll); it is not
 * thread-safe. */
typedef struct fa_server fa_server;

#define FA_SERVER_MAX_SLOTS 64u

/* One finished request, with host steady-clock times in milliseconds since the
 * server was created (fa_server_now_ms). */
typedef struct {
  uint64_t ticket;
  uint32_t session;
  uint32_t slot;
  double submit_ms;    /* fa_server_submit */
  double dispatch_ms;  /* launched on its slot */
  double done_ms;      /* completion seen by fa_server_poll */
} fa_server_done;

/* Up to max_slots slots of configuration *cfg, each admitted only while the
 * device memory taken so far (slots, then sessions) stays within budget_bytes;
 * *n_slots (may be NULL) receives the count.  Errors: FA_E_INVALID_ARG,
 * FA_E_OUT_OF_MEMORY (not even one slot fits), FA_E_CUDA. */
fa_status fa_server_create(fa_server** out, const fa_config* cfg, uint32_t max_slots, uint64_t budget_bytes,
                           uint32_t* n_slots);

/* Synchronizes the device, releases the sessions' meshes and frees the slots. */
void fa_server_destroy(fa_server* server);

/* Open a session: register its mesh (d_pos float[V][3], d_idx uint32[T][3],
 * caller-owned, kept until the session closes) and remember its default output
 * buffers *out (may be NULL: every request then passes its own).  Admission: the
 * registration's device memory must fit the remaining budget.  *session receives
 * the id.  Errors: FA_E_INVALID_ARG (sizes above the slots' maxima),
 * FA_E_OUT_OF_MEMORY (budget), FA_E_CUDA. */
fa_status fa_server_session_open(fa_server* server, const float* d_pos, uint32_t V, const uint32_t* d_idx,
                                 uint32_t T, const fa_frame_out* out, uint32_t* session);

/* Close an idle session (no request queued or running).  Errors: FA_E_INVALID_ARG. */
fa_status fa_server_session_close(fa_server* server, uint32_t session);

/* Queue one view request of a session (params as fa_atlas_frame; out = its
 * outputs, or NULL for the session's default buffers) and dispatch what fits.
 * Checked on the host first.  *ticket (may be NULL) receives its id.
 * Errors: FA_E_INVALID_ARG, FA_E_CUDA. */
fa_status fa_server_submit(fa_server* server, uint32_t session, const fa_frame_params* params,
                           const fa_frame_out* out, uint64_t* ticket);

/* Non-blocking: report up to max_done finished requests into done[], free their
 * slots and dispatch queued requests into them.  *n_done receives the count.  A
 * request's per-frame status is in its outputs' result record.
 * Errors: FA_E_INVALID_ARG, FA_E_CUDA. */
fa_status fa_server_poll(fa_server* server, fa_server_done* done, uint32_t max_done, uint32_t* n_done);

/* Queued and running requests, the most requests that ran at once, and the
 * device bytes taken by slots and sessions (any pointer may be NULL). */
fa_status fa_server_stats(const fa_server* server, uint32_t* queued, uint32_t* running, uint32_t* max_running,
                          uint64_t* used_bytes);

/* The server's clock: milliseconds since creation (host steady clock). */
double fa_server_now_ms(const fa_server* server);

#ifdef __cplusplus
}
#endif

#endif /* FASTATLAS_H_ */
