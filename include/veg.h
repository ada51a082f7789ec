/*
 * veg.h -- C ABI of the GB300 splatting core for Volume Encoding Gaussians
 * (VEG, arXiv 2504.13339).
 *
 * Each 3D Gaussian carries a scalar value v instead of a colour (Sec. 3.2).
 * Rendering (Sec. 3.3) maps v through a transfer function (TF) to colour
 * C(v) and opacity O(v), forms alpha = O(v) * w with a trainable weight w,
 * projects the Gaussian to a 2D screen covariance (EWA splatting), bins the
 * splats into 16x16 pixel tiles, orders each tile's splats by depth and
 * blends them front to back with Eq. 1:
 *     P = sum_i c_i alpha_i prod_{j<i} (1 - alpha_j).
 * The backward pass (Sec. 3.3, "gradients are computed manually") carries
 * dL/dP back through the blend, the TF and the projection.
 *
 * Conventions shared by every entry point
 *   - Memory: every array argument is DEVICE memory owned by the caller,
 *     unless marked "host".  The library never allocates or frees: scratch
 *     memory is a caller-provided workspace sized by the *_workspace_size
 *     query.  Arrays of 4-float records must be 16-byte aligned.
 *   - Streams: all work is enqueued on `stream`; calls return before it
 *     runs.  Inputs must stay valid until the stream reaches the call.
 *   - Errors: a call returns VEG_ERR_INVALID_ARGUMENT before launching
 *     anything when an argument is malformed, VEG_ERR_CUDA when a launch
 *     fails.  Errors found on the device (instance capacity overflow) are
 *     recorded in the workspace header and reported by veg_sync_status.
 *     Nothing aborts, traps or prints.
 *   - Cameras (host structs, copied into kernel parameters): pinhole with
 *     OpenCV axes (x right, y down, z forward), world_to_cam = [R | t]
 *     row-major 3x4; pixel (i, j) is evaluated at the point (i, j) in
 *     pixel units.  The views of one call may differ in image size (except
 *     for the raymarcher, whose views share one size).
 *   - Tiles and pixels of several views: view v's tiles (ceil(W_v/16) x
 *     ceil(H_v/16), row-major) get the global ids off_v + tile with off_v
 *     the tile count of the views before v; per-tile arrays (tile_ranges,
 *     tile_order) are indexed by global id.  Per-pixel arrays hold, view
 *     after view, each view's images of H_v x W_v pixels; for views of one
 *     size these layouts are simply [V][tiles] and [V][images][H][W].
 *   - Gaussians: three float4 arrays of n rows: (mu_x, mu_y, mu_z, v),
 *     (log s_x, log s_y, log s_z, w), (q_w, q_x, q_y, q_z).  v and w are
 *     already activated into [0, 1] (the paper stores them via a sigmoid).
 *   - Transfer functions: n_tf tables of lut_size RGBA float4 entries over
 *     v in [0, 1]: entry k sits at v = k/(lut_size-1), values in between are
 *     linearly interpolated (Sec. 3.3, last paragraph).
 */
#ifndef VEG_H
#define VEG_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum veg_status {
  VEG_OK = 0,
  VEG_ERR_INVALID_ARGUMENT = 1,
  VEG_ERR_CAPACITY = 2,    /* more tile instances than the caller's capacity */
  VEG_ERR_CUDA = 3,        /* a CUDA launch or runtime call failed */
  VEG_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
  VEG_ERR_UNSUPPORTED = 5  /* valid request this build does not handle */
} veg_status;

#define VEG_MAX_VIEWS 64
#define VEG_MAX_IMAGE 16384
#define VEG_TILE 16

typedef struct veg_camera {
  float world_to_cam[12]; /* 3x4 row-major [R | t] */
  float fx, fy, cx, cy;   /* focal lengths and principal point, pixels */
  int32_t width, height;  /* image size, pixels, 1..16384 */
  float near_plane;       /* Gaussians with camera z <= near are culled */
} veg_camera;

typedef struct veg_gaussians {
  const float* mean_v;     /* device [n][4]: mu, v */
  const float* logscale_w; /* device [n][4]: log-scale, w */
  const float* quat;       /* device [n][4]: q_w, q_x, q_y, q_z (any norm > 0) */
  int64_t n;
} veg_gaussians;

typedef struct veg_tf {
  const float* lut; /* device [n_tf][lut_size][4] RGBA, straight alpha */
  int32_t lut_size; /* >= 2 */
  int32_t n_tf;     /* >= 1 */
  /* Optional device int32 [n_views]: view v is composited with table
   * view_tf[v] only, giving one image per view (out [V][1][H][W]); NULL
   * composites every view with every table.  An index outside [0, n_tf)
   * reads as a fully transparent table. */
  const int32_t* view_tf;
} veg_tf;

/* Human-readable name of a status code (static string, never NULL). */
const char* veg_status_string(veg_status status);

/* Number of kernels this library has launched in the process so far
 * (a diagnostic counter, incremented on the host at every launch). */
uint64_t veg_kernel_launches(void);

/*
 * veg_project -- per-Gaussian projection (Sec. 3.3: covariance from S and R,
 * projected to 2D "using the method of Zwicker et al."; TF applied first so
 * that Gaussians mapped to low opacity are culled immediately).
 *
 * For every view v < n_views and Gaussian i < g.n, writes record v*n + i:
 *   splat_geo [V][n][4]: (u_x, u_y, depth, w)  screen mean, camera z, weight
 *   splat_aux [V][n][4]: (a, b, c, v)  conic = inverse 2D covariance
 *       [[a, b], [b, c]] of Sigma' = J W Sigma W^T J^T + 0.3 I
 *   tiles_touched [V][n]: number of 16x16 tiles in the splat's rectangle
 *   rect [V][n][4] int16: tile rectangle (x0, y0, x1, y1), ends exclusive:
 *       the tiles holding a pixel centre inside [u - r, u + r]^2 with
 *       r = ceil(3 sqrt(lambda_max(Sigma')))
 * A culled Gaussian gets tiles_touched = 0 and all-zero records.  Culling:
 * camera z <= near_plane, zero quaternion, det(Sigma') <= 0, empty rectangle,
 * and -- only when cull_tf is non-NULL -- O_t(v) w < 1/255 for every table t
 * of cull_tf (lossless: such a Gaussian can never reach alpha >= 1/255); with
 * cull_tf->view_tf set, view v is tested against table view_tf[v] only.
 * Depth, screen mean, radius, rectangle and the opacity test are evaluated in
 * IEEE float32 with a fixed operation order (no fused multiply-add) so that
 * tile lists are reproducible bit for bit.
 * cams: host [n_views], 1 <= n_views <= VEG_MAX_VIEWS.  cull_tf: host pointer
 * to a descriptor (its lut is device memory) or NULL.
 */
veg_status veg_project(const veg_camera* cams, int32_t n_views, veg_gaussians g,
                       const veg_tf* cull_tf, float* splat_geo, float* splat_aux,
                       int32_t* tiles_touched, int16_t* rect, cudaStream_t stream);

/*
 * veg_project_views -- veg_project where each view shows its own model
 * (a server batching requests for different models into one binning and one
 * compositing call; the paper renders one model per frame, Sec. 3.3).
 * models: host [n_views]; view v projects models[v] (any model, the same
 * one in several views allowed).  n: the record stride, >= every
 * models[v].n.  View v's records are [v*n, v*n + models[v].n), written
 * exactly as veg_project writes them; its records [v*n + models[v].n,
 * (v+1)*n) get tiles_touched = 0 and their other arrays are left untouched
 * (the binning reads nothing else of a record that touches no tile).
 * Downstream calls take n as the Gaussian count: veg_bin_sort and
 * veg_composite_fwd treat the padding records as culled, so each view's
 * image is the one its model renders alone.  Errors as veg_project, and
 * VEG_ERR_INVALID_ARGUMENT when models is NULL or a models[v].n exceeds n.
 */
veg_status veg_project_views(const veg_camera* cams, int32_t n_views,
                             const veg_gaussians* models, int64_t n, const veg_tf* cull_tf,
                             float* splat_geo, float* splat_aux, int32_t* tiles_touched,
                             int16_t* rect, cudaStream_t stream);

/*
 * veg_bin_sort -- tile binning and depth ordering (Sec. 3.3: "the efficient
 * tile-based rasterizer", alpha-blending "in front-to-back order").
 *
 * Produces, for every view and tile, the list of splats touching the tile in
 * increasing (depth, Gaussian index) order; equivalently the stable sort of
 * one key per (Gaussian, tile) pair,
 *     key = (view << (tb + 32)) | (tile << 32) | bits(depth_f32),
 * tb = max(1, ceil(log2(tiles of the largest view))), emitted in Gaussian
 * index order with tiles row-major.  Outputs:
 *   vals [capacity]: record index v*n + i of each instance, sorted
 *   keys [capacity] (optional, may be NULL): the sorted 64-bit keys above
 *   tile_ranges [global tiles][2] int32: [start, end) of each tile's run in
 *       vals ((0, 0) for an empty tile), indexed by global tile id (views
 *       of one size: [V][tiles], tiles = ceil(W/16) * ceil(H/16))
 * The number of instances M is known only on the device; when M > capacity
 * only the first `capacity` instances (in emission order) are binned, the
 * header flag is set and veg_sync_status returns VEG_ERR_CAPACITY.
 * workspace: device, >= veg_bin_sort_workspace_size(...) bytes, 256-byte
 * aligned; its first 256 bytes are a status header read by veg_sync_status.
 * n, capacity >= 0; capacity < 2^31.
 */
veg_status veg_bin_sort_workspace_size(int64_t n, int32_t n_views, int64_t capacity,
                                       int32_t width, int32_t height, size_t* bytes);
veg_status veg_bin_sort(const veg_camera* cams, int32_t n_views, int64_t n,
                        const float* splat_geo, const int32_t* tiles_touched,
                        const int16_t* rect, void* workspace, size_t workspace_bytes,
                        int64_t capacity, uint64_t* keys, uint32_t* vals,
                        int32_t* tile_ranges, cudaStream_t stream);

/*
 * veg_tile_order -- a processing order for the compositing kernels (a
 * scheduling aid of this library; the paper has no counterpart): the
 * indices 0..count-1 of tile_ranges [count][2] (count = the global tiles), the
 * tiles with the longest lists first (bucketed by floor(log2(length)), empty
 * tiles last).  Passing it to veg_composite_fwd/bwd schedules the heaviest
 * tiles first, which shortens the tail of the launch; results do not depend
 * on it.  The order inside a bucket is unspecified (it may differ between
 * calls).  tile_order: device int32 [count], overwritten.
 */
veg_status veg_tile_order(const int32_t* tile_ranges, int64_t count, int32_t* tile_order,
                          cudaStream_t stream);

/*
 * veg_bin_sort_static -- veg_bin_sort without any memory from the caller
 * beyond inputs and outputs.  The paper has no counterpart; this exists for
 * callers that cannot allocate device memory: code that runs while another
 * component holds a CUDA stream capture open (cudaMalloc is not allowed
 * then), real-time render loops that must never enter the driver's
 * allocator, and plug-ins whose host application owns every device
 * allocation.  It runs the same kernels as veg_bin_sort with their scratch in
 * one fixed 16 MiB device array compiled into the library, which every GPU
 * that loads the library holds until the process exits.
 *   Size limit: the scratch needed is about 20 bytes per record (n_views * n)
 *   plus 12 bytes per instance of `capacity` plus 1 KiB per 2048 items of the
 *   larger of the two (e.g. 65,536 records with a capacity of 1,000,000 fit);
 *   a request needing more than 16 MiB returns VEG_ERR_UNSUPPORTED before
 *   anything is launched.  Nothing is allocated or freed, by this library or
 *   any routine it calls.
 *   Outputs: vals, keys (optional), tile_ranges exactly as veg_bin_sort;
 *   n_instances (device int64, optional) receives the instance count M, and
 *   M > capacity means the binning overflowed (only the first `capacity`
 *   instances were binned).  There is no workspace header to pass to
 *   veg_sync_status.
 *   Set-up: the first call in each CUDA context looks up the array's device
 *   address with that context current and keeps it for later calls in the
 *   same context; a device reset (or a primary context released and created
 *   again) makes the next call look it up anew, since the array may then sit
 *   elsewhere.  Make the first call of each context before any stream capture
 *   begins: a lookup needed while `stream` is being captured returns
 *   VEG_ERR_UNSUPPORTED without launching anything.
 *   Sharing: every call on a device uses the same array, which keeps the
 *   previous call's contents; each call writes every scratch word before it
 *   reads it, so no clearing is needed.  Calls whose work overlaps on the GPU
 *   (other streams, other host threads) race on the array: serialise them.
 */
veg_status veg_bin_sort_static(const veg_camera* cams, int32_t n_views, int64_t n,
                               const float* splat_geo, const int32_t* tiles_touched,
                               const int16_t* rect, int64_t capacity, uint64_t* keys,
                               uint32_t* vals, int32_t* tile_ranges, int64_t* n_instances,
                               cudaStream_t stream);

/*
 * veg_radix_lookback_check -- a device check of the binning's radix sort (a
 * diagnostic of this library; the paper has no counterpart).  Sorts of at
 * most 64 chunks of 2048 items (small scenes; larger sorts take three
 * kernels per pass with no waits) run each radix pass as one kernel in which
 * a CTA waits for the digit counts that the CTAs of the earlier chunks
 * publish; every such wait gives up after a bounded number of polls, sets a
 * timeout flag in the workspace header and lets the kernel finish, so a
 * fault in that chain shows as a status, never as a hang.  This call sorts n seeded keys (key i = (i * 2654435761) >> 4,
 * mod 2^32; value i) with that sort, each wait limited to `spins` polls,
 * and copies the sorted keys and values to keys_out and vals_out (device
 * uint32 [n], overwritten).  With starve_first != 0 the first chunk is
 * never taken, so the next chunk's wait runs out: veg_sync_status on the
 * workspace then returns VEG_ERR_TIMEOUT (the outputs are void); otherwise
 * VEG_OK and the stable sort.  workspace: device, 256-byte aligned, >=
 * veg_bin_sort_workspace_size(n, 1, 0, 16, 16) bytes.  1 <= n <= 131072
 * (64 chunks), spins >= 1; else VEG_ERR_INVALID_ARGUMENT.
 */
veg_status veg_radix_lookback_check(void* workspace, size_t workspace_bytes, int64_t n,
                                    int32_t starve_first, int32_t spins, uint32_t* keys_out,
                                    uint32_t* vals_out, cudaStream_t stream);

/*
 * veg_sync_status -- waits for `stream`, then reads the status header of a
 * bin_sort / render workspace.  Writes the instance count M (even when it
 * exceeded the capacity) to *n_instances (host, may be NULL).  Returns
 * VEG_ERR_TIMEOUT if a bounded device-side wait of the last binning gave up
 * (its outputs are then void), VEG_ERR_CAPACITY if the last binning
 * overflowed, VEG_ERR_CUDA if the stream reported an error, else VEG_OK.
 */
veg_status veg_sync_status(const void* workspace, cudaStream_t stream, int64_t* n_instances);

/*
 * veg_composite_fwd -- Eq. 1 per pixel, for n_tf transfer functions at once.
 *
 * For each view, tile, pixel and TF t, walks the tile's list front to back:
 *   G = exp(-1/2 d^T Sigma'^-1 d), d = u - pixel (skip the splat if the
 *       exponent is positive);
 *   (rgb, A) = TF_t(v) by linear interpolation; alpha = min(0.99, A w G);
 *   skip if alpha < 1/255; stop this TF at this pixel if T (1 - alpha) <
 *   1e-4 (that splat not blended); else C += rgb alpha T, T *= 1 - alpha.
 * Writes out [V][n_tf][H][W][4] = (C + T bg, T_final) and n_contrib
 * [V][n_tf][H][W] = 1 + list position of the last blended splat (0 if none)
 * (views of different sizes: view after view, n_tf images of H_v x W_v
 * pixels each; with view_tf one image per view).
 * The scene representation is TF-independent, so one sort serves every TF.
 * tile_order: optional device int32 [global tiles] from veg_tile_order
 * (the order in which tiles are scheduled; NULL = row-major; results do
 * not depend on it).
 * tf_group: TFs composited per pass (1, 2, 4 or 8; 0 = library default, 1;
 * the autotuner of the Python package picks per shape).
 * tile_batch: splats of a tile's list staged per pass through shared memory
 * (128, 256 or 512; 0 = 256; the autotuner picks per shape); results do not
 * depend on it.  The instrumented build (stats) stages 256.
 * splat_shade: optional device float [V][n][2] of Blinn-Phong factors
 * (s_d, s_s) from veg_shade (8-byte aligned); when given, each splat is
 * blended with the colour s_d rgb + s_s of Eq. 2 instead of rgb.  Opacity,
 * skips and termination do not depend on it.  NULL = unshaded.  Shading
 * with stats returns VEG_ERR_UNSUPPORTED.
 * bg: host float[3].  stats: optional device uint64[5] accumulating
 * (visited pixel-splat pairs -- every pair reached before the pixel stops --,
 * pairs walked by the kernel after its culling, pairs above the exponent
 * cutoff -- below it no TF of the group can reach alpha >= 1/255 --, alpha
 * evaluations, blended pairs), NULL to skip the instrumented kernel.  n is the per-view record count used by
 * veg_project.
 */
veg_status veg_composite_fwd(const veg_camera* cams, int32_t n_views, int64_t n,
                             const float* splat_geo, const float* splat_aux,
                             const float* splat_shade, const uint32_t* vals,
                             const int32_t* tile_ranges,
                             const int32_t* tile_order, veg_tf tf, const float* bg,
                             int32_t tf_group, int32_t tile_batch, float* out,
                             int32_t* n_contrib, unsigned long long* stats,
                             cudaStream_t stream);

/*
 * veg_composite_bwd -- manual gradients of the render (Sec. 3.3, backward
 * pass through "the rasterizer", the transfer function and the projection).
 *
 * Given the forward inputs/outputs and dL_dout [V][n_tf][H][W][4] (gradient
 * with respect to (R, G, B, T_final)), walks each pixel's blend back to
 * front and ACCUMULATES (+=) into the caller's gradient arrays, packed like
 * the Gaussians: grad_mean_v [n][4] = (dL/dmu, dL/dv), grad_logscale_w
 * [n][4] = (dL/dlog s, dL/dw), grad_quat [n][4] = dL/dq, summed over views
 * and TFs.  Derivatives are exact: zero through the 0.99 clamp, the skips and
 * the clamped Jacobian entries.  grad2d (optional, may be NULL) receives the
 * per-record screen-space gradients [V][n][8] = (du_x, du_y, da, db, dc, dv,
 * dw, 0) (overwritten).  workspace >= veg_composite_bwd_workspace_size.
 * If grad_mean_v, grad_logscale_w and grad_quat are all NULL, only grad2d
 * (then required) is computed; veg_project_bwd completes the chain.
 * splat_shade: the forward's shading factors or NULL.  When given,
 * grad_shade (device float [V][n][2], 8-byte aligned, overwritten) receives
 * dL/ds_d and dL/ds_s per record, and veg_shade_bwd chains them to the
 * normals, the material coefficients and the means; the colour slopes in dv
 * are scaled by s_d.  Shading with stats returns VEG_ERR_UNSUPPORTED.
 * tf_group (1, 2 or 4; 0 = min(n_tf, 4)) and tile_batch (128, 256 or 512;
 * 0 = 256) as in veg_composite_fwd; results do not depend on them.
 * stats: optional device uint64[7] accumulating (replayed pixel-splat pairs,
 * pairs walked after culling, pairs above the exponent cutoff, alpha
 * evaluations, blended pairs, blended pairs below the 0.99 clamp, pairs with
 * a nonzero screen-space gradient); NULL skips the instrumented kernel.
 */
veg_status veg_composite_bwd_workspace_size(int64_t n, int32_t n_views, size_t* bytes);
veg_status veg_composite_bwd(const veg_camera* cams, int32_t n_views, veg_gaussians g,
                             const float* splat_geo, const float* splat_aux,
                             const float* splat_shade, const int32_t* tiles_touched,
                             const uint32_t* vals,
                             const int32_t* tile_ranges, const int32_t* tile_order, veg_tf tf,
                             const float* bg, int32_t tf_group, int32_t tile_batch,
                             const float* out, const int32_t* n_contrib,
                             const float* dL_dout, void* workspace, size_t workspace_bytes,
                             float* grad_mean_v, float* grad_logscale_w, float* grad_quat,
                             float* grad2d, float* grad_shade, unsigned long long* stats,
                             cudaStream_t stream);

/*
 * veg_project_bwd -- the projection part of the backward pass (Sec. 3.3):
 * chains per-record screen-space gradients grad2d [V][n][8] = (du_x, du_y,
 * da, db, dc, dv, dw, 0) -- as written by veg_composite_bwd -- through the
 * EWA projection, the covariance construction, the scale exponential and the
 * quaternion normalisation, and ACCUMULATES (+=) the sum over views into
 * grad_mean_v, grad_logscale_w and grad_quat [n][4].  Records with
 * tiles_touched == 0 (culled) contribute nothing.  One thread per Gaussian,
 * no atomics: the result is deterministic.
 */
veg_status veg_project_bwd(const veg_camera* cams, int32_t n_views, veg_gaussians g,
                           const int32_t* tiles_touched, const float* grad2d,
                           float* grad_mean_v, float* grad_logscale_w, float* grad_quat,
                           cudaStream_t stream);

/*
 * veg_project_bwd_range -- veg_project_bwd for the Gaussians [first,
 * first + count) only (0 <= first, 0 <= count, first + count <= g.n; else
 * VEG_ERR_INVALID_ARGUMENT).  All arrays keep their full-model layout
 * (grad2d [V][g.n][8], tiles_touched [V][g.n], gradients [g.n][4]); rows
 * outside the range are neither read nor written.  Each Gaussian's result is
 * the same as in the whole-model call, so a backward split into ranges is
 * bit-identical to one call.  A data-parallel step uses it to start the
 * gradient all-reduce of one range while the next range is still computed.
 */
veg_status veg_project_bwd_range(const veg_camera* cams, int32_t n_views, veg_gaussians g,
                                 const int32_t* tiles_touched, const float* grad2d,
                                 int64_t first, int64_t count, float* grad_mean_v,
                                 float* grad_logscale_w, float* grad_quat, cudaStream_t stream);

/*
 * veg_shade -- Blinn-Phong factors of Eq. 2-3 per view and Gaussian (Sec. 3.3,
 * "Phong shading").  For view v and Gaussian i, with n = normal / |normal|,
 * l the unit light direction of the view (world space, toward the light; a
 * headlight is the camera's backward optical axis), e the unit vector from
 * the mean toward the camera centre and h = (e + l) / |e + l|:
 *   s_d = k_a + k_d |n.l|,   s_s = k_s |n.h|^beta if |n.l| > 0 else 0,
 * so that the shaded colour of Eq. 2 is s_d C(v) + s_s (white specular).
 * mean_v [n][4] (mu, v) as for veg_project; normal_beta [n][4] = (normal,
 * beta); k_ads [n][4] = (k_a, k_d, k_s, unused): device, 16-byte aligned.
 * light_dirs: host float [n_views][3], normalised here (zero length is
 * VEG_ERR_INVALID_ARGUMENT).  splat_shade: device float [n_views][n][2]
 * (s_d, s_s), overwritten, 8-byte aligned.  One launch, no atomics.
 */
veg_status veg_shade(const veg_camera* cams, int32_t n_views, const float* mean_v, int64_t n,
                     const float* normal_beta, const float* k_ads, const float* light_dirs,
                     float* splat_shade, cudaStream_t stream);

/*
 * veg_shade_bwd -- the backward pass of Eq. 2-3 (Sec. 4.2 trains the normals
 * and lighting coefficients): chains grad_shade [n_views][n][2] =
 * (dL/ds_d, dL/ds_s), as
 * written by veg_composite_bwd, through veg_shade and ACCUMULATES (+=) the sum
 * over views into grad_mean_v [n][4] (dL/dmu in xyz; w untouched),
 * grad_normal_beta [n][4] = (dL/dnormal, dL/dbeta) and grad_k_ads [n][4] =
 * (dL/dk_a, dL/dk_d, dL/dk_s, untouched).  Derivatives of |.| use its sign
 * (0 at 0).  Records with tiles_touched == 0 contribute nothing.  One thread
 * per Gaussian, no atomics: deterministic.  Same layouts and alignment as
 * veg_shade.
 */
veg_status veg_shade_bwd(const veg_camera* cams, int32_t n_views, const float* mean_v, int64_t n,
                         const float* normal_beta, const float* k_ads, const float* light_dirs,
                         const int32_t* tiles_touched, const float* grad_shade,
                         float* grad_mean_v, float* grad_normal_beta, float* grad_k_ads,
                         cudaStream_t stream);

/*
 * veg_l1_loss -- the L1 part of the training loss (Sec. 4.2:
 * (1 - lambda) L1 + lambda L_SSIM): loss = mean |out.rgb - target.rgb| over
 * n_records RGBA records (the fourth channel ignored), and
 * grad = dloss/dout (sign(out - target) / (3 n_records) on RGB, 0 on the
 * fourth channel; sign(0) = 0).  loss: device float, overwritten.
 * workspace >= veg_l1_loss_workspace_size bytes; the sum is reduced in a
 * fixed order, so the result is deterministic.
 */
veg_status veg_l1_loss_workspace_size(size_t* bytes);
veg_status veg_l1_loss(const float* out, const float* target, int64_t n_records, float* grad,
                       float* loss, void* workspace, size_t workspace_bytes,
                       cudaStream_t stream);

/*
 * veg_l1_ssim_loss -- the training image loss of Sec. 4.2,
 *   loss = (1 - lambda) L1 + lambda (1 - SSIM),  lambda = 0.2 in the paper,
 * over n_images RGBA images [n_images][height][width][4] (the fourth channel
 * takes no part).  L1 = mean |out - target| over RGB; SSIM (Wang et al.
 * 2004) = mean over RGB pixels of the structural similarity index under an
 * 11 x 11 Gaussian window (sigma 1.5, normalised, zero padding at the image
 * border) with C1 = 0.01^2, C2 = 0.03^2.  Writes grad = dloss/dout (same
 * shape, 0 on the fourth channel; sign(0) = 0 for the L1 part) and the device
 * float[3] loss = (loss, L1, SSIM).  workspace >=
 * veg_l1_ssim_loss_workspace_size bytes (16-byte aligned; it holds the
 * per-tile sums and the per-pixel partial derivatives of S, 36 B per pixel
 * and image); per-tile sums are reduced in a fixed order, so the result is
 * deterministic.  Three launches.  n_images <=
 * 65535; lambda in [0, 1].
 */
veg_status veg_l1_ssim_loss_workspace_size(int64_t n_images, int32_t height, int32_t width,
                                           size_t* bytes);
veg_status veg_l1_ssim_loss(const float* out, const float* target, int64_t n_images,
                            int32_t height, int32_t width, float lambda, float* grad, float* loss,
                            void* workspace, size_t workspace_bytes, cudaStream_t stream);

/*
 * veg_adam_step -- one Adam step (Kingma and Ba, bias-corrected) on the
 * Gaussians' stored parameters, the optimiser of the paper's training
 * (Sec. 4.2, 5.1).  Five packed device arrays [n][4], each optional (NULL
 * param = skipped): 0 raw (mu, v), 1 raw (log-scale, w), 2 quaternion,
 * 3 (normal, beta), 4 (k_a, k_d, k_s, -).  v and w are stored raw and
 * activated by the logistic sigmoid (Sec. 3.3); every other value is used as
 * stored.  grad[a] holds dL/d(rendered value) (as accumulated by
 * veg_composite_bwd and veg_shade_bwd); for the sigmoid components the raw
 * gradient g s (1 - s) is formed here.  exp_avg / exp_avg_sq are the moment
 * arrays (zero before step 1).  rendered[0], rendered[1] (optional) receive
 * the activated (mu, sigmoid(v)) and (log-scale, sigmoid(w)) for the next
 * render.  lr: host float[20], per array and component.  step >= 1.  All
 * arrays 16-byte aligned.  One launch.
 */
typedef struct veg_adam_arrays {
  float* param[5];
  const float* grad[5];
  float* exp_avg[5];
  float* exp_avg_sq[5];
  float* rendered[2];
} veg_adam_arrays;
veg_status veg_adam_step(const veg_adam_arrays* arrays, int64_t n, const float* lr, float beta1,
                         float beta2, float eps, int32_t step, cudaStream_t stream);

/*
 * veg_adam_step_counted -- veg_adam_step with the step number kept on the
 * device, so that a captured CUDA graph can replay the optimiser: `counter`
 * (device, 16-byte aligned, caller-owned, zeroed before the first step)
 * holds the steps taken; each call advances it by one (one single-thread
 * launch) and takes the step with t = the new count, its bias corrections
 * computed in double on the device as veg_adam_step computes them on the
 * host.  Two launches (one with n = 0).
 */
typedef struct veg_adam_counter {
  int64_t step;
  float inv_bc1;      /* 1 / (1 - beta1^t) of the last step */
  float inv_sqrt_bc2; /* 1 / sqrt(1 - beta2^t) of the last step */
} veg_adam_counter;
veg_status veg_adam_step_counted(const veg_adam_arrays* arrays, int64_t n, const float* lr,
                                 float beta1, float beta2, float eps, veg_adam_counter* counter,
                                 cudaStream_t stream);

/*
 * veg_grad_stats_accumulate -- the densification statistic of Sec. 4.2
 * (3D Gaussian splatting's "view-space positional gradient"): for every view
 * v and Gaussian i with tiles_touched[v][i] > 0, adds |(g_x W/2, g_y H/2)| to
 * accum[i] and 1 to count[i], where (g_x, g_y) = dL/du are the first two
 * values of grad2d [V][n][8] as written by veg_composite_bwd (the screen-mean
 * gradient in pixels, W/2 and H/2 converting it to normalised device units).
 * Float32 with every product, sum and square root rounded separately, views
 * in order, one thread per Gaussian: deterministic.  accum float[n], count
 * int32[n], device, accumulated.
 */
veg_status veg_grad_stats_accumulate(const float* grad2d, const int32_t* tiles_touched,
                                     int64_t n, int32_t n_views, int32_t width, int32_t height,
                                     float* accum, int32_t* count, cudaStream_t stream);

/*
 * veg_densify -- one clone / split / prune pass (Sec. 4.2, following 3D
 * Gaussian splatting).  Per Gaussian i, in float32 against the thresholds of
 * cfg (prepared by the caller):
 *   prune  if raw w < raw_weight_threshold  (the paper's w < 0.005 on the
 *          sigmoid-activated weight);
 *   else, if accum[i] / count[i] >= grad_threshold (0 when count is 0):
 *     split if max(log-scale) > log_size_threshold (ln(0.01 x scene extent)),
 *     clone otherwise;
 *   else keep.
 * Outputs, in input order, into `out` (arrays of capacity out_capacity >= 2n
 * rows): keep -> the Gaussian with its Adam moments; clone -> the Gaussian
 * with its moments, then a copy with zero moments; split -> two children
 * mu + R(q) diag(exp(log-scale)) z_j (z = split_normals [n][2][3], standard
 * normal samples supplied by the caller), log-scale - log_split_factor,
 * every other value copied, zero moments; prune -> nothing.  `in` and `out`
 * use param / exp_avg / exp_avg_sq of veg_adam_arrays (grad ignored; a NULL
 * param array is skipped; arrays 0-2 required); out->rendered[0..1], if
 * given, receive the activated (mu, sigmoid(v)) and (log-scale, sigmoid(w)).
 * *n_out (device int64) receives the output count; action (optional device
 * int32[n]) the decision (0 prune, 1 keep, 2 clone, 3 split).  workspace >=
 * veg_densify_workspace_size bytes, 256-byte aligned.  Three launches.
 */
typedef struct veg_density_config {
  float grad_threshold;        /* 0.0002 */
  float log_size_threshold;    /* ln(0.01 x scene extent) */
  float raw_weight_threshold;  /* logit(0.005) */
  float log_split_factor;      /* ln(1.6) */
} veg_density_config;
veg_status veg_densify_workspace_size(int64_t n, size_t* bytes);
veg_status veg_densify(const veg_adam_arrays* in, int64_t n, const float* accum,
                       const int32_t* count, const float* split_normals, veg_density_config cfg,
                       const veg_adam_arrays* out, int64_t out_capacity, int64_t* n_out,
                       int32_t* action, void* workspace, size_t workspace_bytes,
                       cudaStream_t stream);

/*
 * veg_volume_prepare -- packs a scalar volume (the gridded data of Sec. 3.1
 * and 4.1) for veg_raymarch: volume
 * float [R][R][R] (x fastest) of vertex values at x_i = -1 + 2i/(R-1) on
 * each axis of [-1,1]^3; vol4 float4 [R][R][R] receives (value, dv/dx,
 * dv/dy, dv/dz) with central-difference gradients ((v[i+1] - v[i-1]) / 2h,
 * one-sided on the boundary faces; h = 2/(R-1)).  2 <= R <= 2048; vol4
 * 16-byte aligned.  One launch.
 */
veg_status veg_volume_prepare(const float* volume, int32_t resolution, float* vol4,
                              cudaStream_t stream);

/*
 * veg_raymarch -- emission-absorption raymarching of the prepared volume,
 * the renderer of the paper's ground-truth images (Sec. 4.2, 5.1: raymarched
 * with an emission-absorption model, Blinn-Phong shaded with a headlight).
 * Per pixel of every view (camera model of veg_project): the ray from the
 * camera centre through the pixel, clipped to [-1,1]^3 and t >= near, is
 * sampled at t0 + (k + 1/2) step for k < floor((t1 - t0) / step); a sample's
 * value v and gradient are trilinear blends of vol4; its opacity is
 * alpha = 1 - (1 - A(v))^(step / h) (A per unit distance h, the grid
 * spacing) and its colour C(v), both from the tables of `tf` (linear
 * interpolation as in veg_composite_fwd); with `material`, the colour is
 * (k_a + k_d |n.l|) C + k_s |n.h|^beta with n the normalised gradient
 * (k_a C where the gradient vanishes), l the headlight (camera backward axis)
 * and h the half vector of l and the view direction.  Front-to-back
 * compositing stops once T < 1e-4.  out [V][n_tf][H][W][4] = (C + T bg, T)
 * (one image per view with tf.view_tf).  bg host float[3] or NULL (black).
 * stats: optional device uint64[2] accumulating (samples taken per ray and
 * table group, table evaluations); NULL skips the instrumented kernel.
 */
typedef struct veg_material {
  float ka, kd, ks, beta;
} veg_material;
veg_status veg_raymarch(const veg_camera* cams, int32_t n_views, const float* vol4,
                        int32_t resolution, veg_tf tf, float step, const veg_material* material,
                        const float* bg, float* out, unsigned long long* stats,
                        cudaStream_t stream);

/*
 * veg_raymarch_cells -- empty-space acceleration for veg_raymarch_masked
 * (not part of the paper's method; it only skips work): the vertex cells of
 * the prepared volume are grouped into macrocells of cell^3 (cell a power
 * of two, 1..64; ceil((R-1)/cell) macrocells per axis, x fastest), and
 * mask[macrocell] bit t (t < 32) is set when table t of `tf` can give a
 * sample in the macrocell a positive opacity: some table entry that values
 * within the macrocell's vertex range (widened by 1e-6, plus one entry on
 * each side) interpolate between has a positive opacity.  Every bit is set
 * for a macrocell holding a NaN vertex, and for every macrocell when
 * tf.n_tf > 32.  veg_raymarch_cells_count gives the number of macrocells
 * (the length of `mask`, device uint32).  One launch.
 */
veg_status veg_raymarch_cells_count(int32_t resolution, int32_t cell, int64_t* count);
veg_status veg_raymarch_cells(const float* vol4, int32_t resolution, veg_tf tf, int32_t cell,
                              uint32_t* mask, cudaStream_t stream);

/*
 * veg_raymarch_masked -- veg_raymarch with an empty-space mask from
 * veg_raymarch_cells (the same vol4, tf tables and cell; NULL = none): a
 * sample whose macrocell has no positive opacity for any table of its group
 * still compositing is skipped.  Such a sample has opacity exactly 0 in all
 * of them and leaves colour and transmittance unchanged, so the images are
 * identical to veg_raymarch's.  stats: optional device uint64[3] with a
 * mask ((samples taken, table evaluations, samples skipped); samples taken
 * excludes skipped ones), uint64[2] without.
 */
veg_status veg_raymarch_masked(const veg_camera* cams, int32_t n_views, const float* vol4,
                               int32_t resolution, veg_tf tf, float step,
                               const veg_material* material, const float* bg,
                               const uint32_t* cell_mask, int32_t cell, float* out,
                               unsigned long long* stats, cudaStream_t stream);

/*
 * veg_train_step -- one opacity-guided training iteration (Sec. 4.2) issued
 * from native code: veg_project (culled by the chosen table) ->
 * veg_shade (headlight of the chosen view, if lit) -> veg_bin_sort ->
 * veg_tile_order -> veg_composite_fwd -> veg_l1_ssim_loss against
 * targets[view][map] -> zeroing of the gradients -> veg_composite_bwd
 * (full chain) -> veg_shade_bwd (if lit) -> veg_grad_stats_accumulate (if
 * stat_accum is given and accumulate_stats) -> veg_adam_step (if
 * adam_step >= 1).  Every buffer is the caller's (the library allocates
 * nothing); the arrays and sizes follow the entry points named above.  No
 * host synchronisation: instance-capacity overflow is reported later by
 * veg_sync_status on binsort_ws.  Returns the first failing status.
 */
typedef struct veg_train_args {
  /* model: raw parameters, gradients, Adam moments ([n][4] each; arrays 3,
   * 4 may be NULL when unlit) and the rendered (activated) arrays */
  float* raw[5];
  float* grad[5];
  float* exp_avg[5];
  float* exp_avg_sq[5];
  float* mean_v;
  float* logscale_w;
  int64_t n;
  /* training set: host cameras and headlights, device tables and targets */
  const veg_camera* cams;
  int32_t n_cams;
  const float* light_dirs; /* host [n_cams][3] */
  const float* luts;       /* device [n_maps][lut_size][4] */
  int32_t lut_size, n_maps;
  const float* targets;    /* device [n_cams][n_maps][H][W][4] */
  float bg[3];
  float lambda;            /* SSIM weight of the loss */
  float lr[20];
  float beta1, beta2, eps;
  int32_t lit;
  int32_t tf_group;
  /* render buffers for one view of n records */
  float* splat_geo;
  float* splat_aux;
  int32_t* tiles_touched;
  int16_t* rect;
  float* splat_shade;      /* [n][2], if lit */
  float* grad_shade;       /* [n][2], if lit */
  void* binsort_ws;
  size_t binsort_ws_bytes;
  int64_t capacity;
  uint32_t* vals;
  int32_t* tile_ranges;
  int32_t* tile_order;
  float* out;              /* [H][W][4] */
  int32_t* n_contrib;
  float* loss_grad;        /* [H][W][4] */
  float* grad2d;           /* [n][8] */
  float* loss;             /* device float[3] */
  void* loss_ws;
  size_t loss_ws_bytes;
  float* stat_accum;       /* optional densification statistic */
  int32_t* stat_count;
} veg_train_args;
veg_status veg_train_step(const veg_train_args* args, int32_t view, int32_t map,
                          int32_t adam_step, int32_t accumulate_stats, cudaStream_t stream);

/*
 * veg_render -- the forward render of Sec. 3.3 in one call: projection with
 * the TF cull (veg_project), tile binning and depth sort (veg_bin_sort), the
 * longest-first tile schedule (veg_tile_order) and Eq. 1 compositing
 * (veg_composite_fwd), all scratch in `workspace` (device, 256-byte
 * aligned, >= veg_render_workspace_size bytes; width and height there are
 * the largest view's).  tf_group: TFs per compositing pass, 0 = the
 * library's default (1), else 1, 2, 4 or 8; results do not depend on it.
 * Outputs out and n_contrib as veg_composite_fwd (caller-owned device
 * memory, overwritten).  Overflow of `capacity` is reported by
 * veg_sync_status on the same workspace.  Returns VEG_ERR_INVALID_ARGUMENT
 * before launching anything for malformed arguments or a workspace too
 * small for these views.
 */
veg_status veg_render_workspace_size(int64_t n, int32_t n_views, int64_t capacity,
                                     int32_t width, int32_t height, size_t* bytes);
veg_status veg_render(const veg_camera* cams, int32_t n_views, veg_gaussians g, veg_tf tf,
                      const float* bg, int32_t tf_group, int64_t capacity, void* workspace,
                      size_t workspace_bytes, float* out, int32_t* n_contrib,
                      cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* VEG_H */
