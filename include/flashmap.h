/*
 * flashmap.h -- C ABI of the GB300 (sm_103a) radiomic spatial-mapping library
 * (libflashmap.so).
 *
 * What the library computes.  Spatial mapping (paper: Introduction; "Software
 * design and extraction modes") returns, for every voxel v of a masked volume
 * of interest (VOI), the radiomic features of the image restricted to the
 * local neighbourhood of v, as maps aligned with the source image.  Here:
 *
 *   V(v)      = { u : max(|ux-vx|, |uy-vy|, |uz-vz|) <= r } n image n VOI
 *   map_f(v)  = feature f of the gray levels / intensities in V(v)
 *
 * with one discretisation of the whole VOI (fixed bin number or fixed bin
 * width; paper: "Hybrid CUDA backend implementation", where discretisation is
 * a preprocessing step).  The 93 features are the spatial benchmark set of
 * Table 2: first order 18, GLCM 24, GLRLM 16, GLSZM 16, NGLDM (GLDM) 14,
 * NGTDM 5, with the IBSI definitions the paper's backends follow.  GLCM and
 * GLRLM features are computed per direction (13 directions, GLCM offset
 * delta * d) and averaged over the directions whose matrix is not empty;
 * zones are 26-connected; dependences use alpha = 0 and distance 1.
 *
 * Conventions shared by every entry point.
 *   - Every call returns an fr_status; nothing aborts, throws or prints.
 *   - Volumes are C-contiguous [nz][ny][nx] (x fastest).  Images are int16,
 *     masks uint8 (nonzero = inside the VOI).
 *   - The caller owns images, masks and outputs; a plan owns its device
 *     scratch and frees it in fr_map_destroy.
 *   - "Device pointer" means memory of the plan's CUDA device (cudaMalloc,
 *     or a torch tensor's data_ptr()).  Streams are cudaStream_t values
 *     passed as fr_stream_t (NULL = the legacy default stream).
 *   - Output layout: out[row][k] float32, row-major [n_rows][n_voi].  Column
 *     k is the k-th VOI voxel in increasing linear index (z, then y, then x);
 *     rows are the selected features in increasing feature id.  Undefined
 *     values (0/0, single gray level where a second is needed, ...) are NaN.
 *   - A plan is used from one stream at a time; calls on one plan must not
 *     overlap on the device.
 *   - Errors that happen on the device (a level count above 255 under fixed
 *     bin width, a bounded wait that ran out) are recorded in a plan-owned
 *     status word; fr_map_sync_status() waits for the plan's work and
 *     returns it.  Output contents are undefined after such an error.
 */
#ifndef FLASHMAP_H
#define FLASHMAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* fr_stream_t; /* = cudaStream_t */

typedef enum fr_status {
  FR_OK = 0,
  FR_ERR_INVALID_ARG = 1,     /* a parameter is out of range or a pointer is NULL */
  FR_ERR_EMPTY_MASK = 2,      /* the mask selects no voxel */
  FR_ERR_TOO_MANY_LEVELS = 3, /* discretisation needs more than 255 gray levels */
  FR_ERR_OOM = 4,             /* a device or host allocation failed */
  FR_ERR_CUDA = 5,            /* a CUDA runtime or driver call failed */
  FR_ERR_TIMEOUT = 6,         /* a bounded device wait ran out */
  FR_ERR_UNSUPPORTED = 7,     /* no usable sm_103a device, or a size beyond a limit */
  FR_ERR_MISMATCH = 8,        /* arguments disagree with the plan (debug calls) */
  FR_ERR_IO = 9               /* a file could not be created or written (HDF5 drain) */
} fr_status;

enum { FR_FBN = 0, FR_FBW = 1 };                             /* discretisation */
enum { FR_ANCHOR_VOI_MIN = 0, FR_ANCHOR_ZERO_FLOOR = 1 };    /* FBW bin anchor  */
/* Texture aggregation over the 13 directions (IBSI 3D:avg / 3D:mrg; the
 * paper's IBSI configurations fix it per family, "IBSI compliance tests").
 * AVERAGE: GLCM and GLRLM features per direction, mean over the non-empty
 * directions.  MERGED: the 13 directional matrices are summed first and the
 * features taken once; GLRLM RunPercentage then divides by 13 N_v (each
 * voxel lies on one run per direction).  GLSZM, GLDM and NGTDM do not
 * depend on a direction. */
enum { FR_AGG_AVERAGE = 0, FR_AGG_MERGED = 1 };
/* 101 features (Table 2's default spatial column): ids 0..92 are the 93-map
 * benchmark set, ids 93..100 the IBSI features completing the default set
 * (see FR_EXTRAS_BEGIN).  fr_map_params_init selects the 93 benchmark maps. */
enum { FR_NUM_FEATURES = 101, FR_NUM_BENCH_FEATURES = 93, FR_NUM_DIRECTIONS = 13,
       FR_MAX_RADIUS = 7 };

/* Feature id ranges (ids are stable; names from fr_feature_name). */
enum {
  FR_FIRSTORDER_BEGIN = 0, FR_GLCM_BEGIN = 18, FR_GLRLM_BEGIN = 42,
  FR_GLSZM_BEGIN = 58, FR_GLDM_BEGIN = 74, FR_NGTDM_BEGIN = 88,
  /* 93..95 statistics: median absolute deviation, coefficient of variation,
   * quartile coefficient of dispersion; 96..97 GLCM: sum variance,
   * dissimilarity; 98..100 NGLDM: grey level non-uniformity normalised,
   * dependence count percentage, dependence count energy (IBSI) */
  FR_EXTRAS_BEGIN = 93, FR_FEATURES_END = 101
};
/* Scalar extraction reports one statistic more than mapping (Table 2:
 * statistics 22 in the scalar benchmark column, 21 in the default spatial
 * column; scalar benchmark total 102 = the 101 map features + 1): id 101,
 * the standard deviation sqrt(m2) of the raw intensities (population, the
 * square root of firstorder_Variance).  It has no map: fr_map_plan rejects a
 * mask that selects it; fr_scalar_plan accepts ids 0..101. */
enum { FR_SCALAR_STDDEV = 101, FR_NUM_SCALAR_FEATURES = 102 };

/* Mapping parameters (the paper's settings object: feature families,
 * discretisation, VOI handling; "Software design and extraction modes"). */
typedef struct fr_map_params {
  int32_t nx, ny, nz;       /* volume extents (each >= 1)                         */
  double spacing[3];        /* voxel spacing in mm (x, y, z); TotalEnergy only    */
  int32_t disc_mode;        /* FR_FBN or FR_FBW                                   */
  int32_t bin_count;        /* FBN: Ng in 1..255                                  */
  double bin_width;         /* FBW: w > 0; Ng = floor((xmax - anchor)/w) + 1      */
  int32_t fbw_anchor;       /* FR_ANCHOR_VOI_MIN (xmin) or FR_ANCHOR_ZERO_FLOOR   */
  int32_t kernel_radius;    /* r in 1..7: window side 2r+1                        */
  int32_t glcm_distance;    /* delta >= 1: GLCM pairs (u, u + delta*d)            */
  uint64_t feature_mask[2]; /* bit f (word f/64, bit f%64) selects feature id f   */
  int32_t kurtosis_excess;  /* 1: m4/m2^2 - 3 (IBSI; default); 0: m4/m2^2         */
  int32_t device;           /* CUDA device ordinal                                */
  int32_t mask_on_device;   /* 1: the mask pointer is a device pointer; 0: host   */
  int32_t aggregation;      /* FR_AGG_AVERAGE (default) or FR_AGG_MERGED          */
  /* Intensity range of the discretisation.  0 (default): the VOI's own
   * minimum and maximum.  1: [range_min, range_max] as given, with each
   * intensity clamped to it before its gray level is taken (raw intensities
   * are used unclamped elsewhere).  A z-slab of one volume planned on its
   * own (sharding across GPUs, section "Multi-GPU" of the design) passes the
   * whole VOI's range, so every slab discretises as the whole volume does
   * and the slabs' maps reassemble the whole volume's maps exactly. */
  int32_t range_given;      /* 0 or 1                                             */
  int32_t range_min;        /* int16 value, <= range_max (range_given = 1)        */
  int32_t range_max;        /* int16 value                                        */
} fr_map_params;

/* Launch shape of the mapping kernel (the autotuner's knobs).  Zero fields
 * take built-in defaults: bricks of 16 x 8 x 8 voxels where every kernel
 * radius is at most 3 and the plan maps at least 100,000 VOI voxels (counted
 * from host masks; a device mask counts its whole volume), else 8 x 4 x 4;
 * 16 voxels per work item, 16 consumer warps, 1 stage, as many CTAs per SM
 * as fit.  A server takes the large bricks up to radius 3. */
typedef struct fr_tune {
  int32_t brick_x, brick_y, brick_z; /* voxels per brick; brick_x % 4 == 0      */
  int32_t voxels_per_item;           /* work-queue granularity (1..1024)       */
  int32_t consumer_warps;            /* warps per CTA that map voxels (1..16)  */
  int32_t stages;                    /* TMA halo buffers per CTA (1..4)        */
  int32_t ctas_per_sm;               /* persistent CTAs per SM (0 = max fit)   */
} fr_tune;

typedef struct fr_plan fr_plan;
typedef struct fr_batch fr_batch;

/* Fill p with defaults for an nx * ny * nz volume: FBN 16, r = 1, delta = 1,
 * all 93 features, unit spacing, excess kurtosis, device 0, host mask. */
void fr_map_params_init(fr_map_params* p, int32_t nx, int32_t ny, int32_t nz);

/* Plan a mapping for one mask: builds on the device the VOI voxel list (z-major),
 * the brick schedule and the work queue, and allocates the scratch the runs
 * need.  Synchronous.  mask: host or device pointer per p->mask_on_device.
 * tune may be NULL.  On success *out owns everything; free it with
 * fr_map_destroy.  Errors: INVALID_ARG, EMPTY_MASK, OOM, CUDA, UNSUPPORTED. */
fr_status fr_map_plan(const fr_map_params* p, const uint8_t* mask,
                      const fr_tune* tune, fr_plan** out);

/* Map one image (device pointer, [nz][ny][nx] int16) into out (device pointer,
 * float32 [n_rows][n_voi]).  Asynchronous on stream s: discretisation,
 * packing and the mapping kernel are queued; no host synchronisation. */
fr_status fr_map_run(fr_plan* plan, const int16_t* image, float* out,
                     fr_stream_t s);

/* Same as fr_map_run with HOST image and output buffers: copies the image to
 * the device, maps it and copies the maps back, then waits for the stream.
 * Pinned host memory makes the copies asynchronous DMA.  Device staging
 * buffers are allocated by the plan on first use.  Returns the device status
 * of the run (as fr_map_sync_status would). */
fr_status fr_map_run_host(fr_plan* plan, const int16_t* image_host,
                          float* out_host, fr_stream_t s);

/* Wait for the plan's queued work and return the device-side status of the
 * last run (FR_OK, FR_ERR_TOO_MANY_LEVELS or FR_ERR_TIMEOUT) or FR_ERR_CUDA. */
fr_status fr_map_sync_status(fr_plan* plan);

/* Sizes of a plan: VOI voxel count (= output columns), output rows, and the
 * device bytes the plan holds.  Any pointer may be NULL. */
fr_status fr_plan_query(const fr_plan* plan, int64_t* n_voi, int32_t* n_rows,
                        size_t* device_bytes);

/* Linear voxel index (z*ny + y)*nx + x of every output column, into idx
 * (device pointer, int32 [n_voi]).  Asynchronous on s. */
fr_status fr_plan_voxel_index(const fr_plan* plan, int32_t* idx, fr_stream_t s);

/* After a run: the discretised gray levels (device pointer, uint8
 * [nz][ny][nx], 0 outside the VOI), and into host ints the level count Ng and
 * the VOI intensity range.  Synchronous.  Any pointer may be NULL. */
fr_status fr_plan_levels(fr_plan* plan, uint8_t* levels, int32_t* ng,
                         int32_t* xmin, int32_t* xmax);

/* Scatter maps to dense volumes: dense[row][z][y][x] = out[row][k] at VOI
 * voxels, NaN elsewhere (the paper's maps aligned with the source image).
 * Device pointers; asynchronous on s. */
fr_status fr_scatter_dense(const fr_plan* plan, const float* out, float* dense,
                           fr_stream_t s);

/* Debug: the integer texture matrices the mapping kernel builds, for n
 * output columns cols[] (host int32) of an image (device pointer).  ng must
 * equal the level count of this image's discretisation (else MISMATCH).  One
 * record of fr_debug_record_ints(plan, ng) int32 per column is written to
 * rec (device pointer), in this order:
 *   [0..3]   ng, s = 2r+1, w = s^3, N_v
 *   hist     [ng]            voxels of each level in V(v)
 *   glcm     [13][ng][ng]    symmetric co-occurrence counts per direction
 *   glrlm    [13][ng][s]     runs of level i and length j+1 per direction
 *   glszm    [ng][w]         zones of level i and size j+1
 *   gldm     [ng][27]        voxels of level i with j equal 26-neighbours
 *   ngtdm_n  [ng]            voxels of level i with at least one neighbour
 *   ngtdm_sl [ng] int64      s_i * lcm(1..26), exact (8-byte aligned)
 * Direction d is the d-th vector (dz, dy, dx) of {-1,0,1}^3 that is
 * lexicographically greater than (0, 0, 0).  Synchronous. */
int64_t fr_debug_record_ints(const fr_plan* plan, int32_t ng);
fr_status fr_debug_matrices(fr_plan* plan, const int16_t* image,
                            const int32_t* cols, int32_t n, int32_t ng,
                            int32_t* rec, fr_stream_t s);

/* Testing hook of failure detection (no GPU fault is made): every device
 * wait of the mapping kernel is bounded in time, and a wait that runs out
 * records FR_ERR_TIMEOUT in the plan's status word and makes every CTA leave
 * (after its own copies in flight have landed).  After this call, runs of
 * the plan bound each wait by wait_limit_ns (0 = the default, 10 s) and,
 * when item >= 0, the feeder leaves the halo buffer of work item `item`
 * unfilled: it issues no copy for it and never completes the buffer's
 * barrier, so the waits on that buffer run out and fr_map_sync_status
 * returns FR_ERR_TIMEOUT; the outputs of such a run are undefined.  item =
 * -1 restores normal runs; the status word is cleared at the start of every
 * run, so the next normal run is unaffected.  Errors: INVALID_ARG for item
 * outside -1 .. (work items - 1) or a negative limit.  Host-side only; takes
 * effect from the next fr_map_run. */
fr_status fr_debug_wait_fault(fr_plan* plan, int32_t item, int64_t wait_limit_ns);

/* Device time in milliseconds of the mapping kernel of the plan's last run,
 * measured by CUDA events the library records on the launching stream
 * immediately before and after that kernel (the discretisation and packing
 * kernels before it are excluded).  Waits for the run.  Errors: INVALID_ARG
 * before any run. */
fr_status fr_plan_last_kernel_ms(fr_plan* plan, float* ms);

/* Free a plan (NULL is a no-op).  Waits for the plan's device work. */
void fr_map_destroy(fr_plan* plan);

/* Batched mapping (continuous-batching building block): n independent
 * (params, mask) pairs share one persistent kernel launch fed by one device
 * work queue of ragged items, launched as a captured CUDA graph.  params[i]
 * and masks[i] as for fr_map_plan (all on one device).  tune may be NULL. */
fr_status fr_batch_plan(const fr_map_params* params, const uint8_t* const* masks,
                        int32_t n, const fr_tune* tune, fr_batch** out);
fr_status fr_batch_query(const fr_batch* b, int32_t i, int64_t* n_voi,
                         int32_t* n_rows);
/* images[i] / outs[i]: device pointers, as for fr_map_run.  The pointer
 * arrays themselves are host arrays.  Asynchronous on s. */
fr_status fr_batch_run(fr_batch* b, const int16_t* const* images,
                       float* const* outs, fr_stream_t s);
fr_status fr_batch_sync_status(fr_batch* b);
/* As fr_plan_last_kernel_ms, for the batch's persistent kernel. */
fr_status fr_batch_last_kernel_ms(fr_batch* b, float* ms);
void fr_batch_destroy(fr_batch* b);

/* Scalar extraction (the paper's other extraction mode, "Software design and
 * extraction modes"): the selected features of the whole VOI, one value per
 * feature -- the map value of a window that covers every VOI voxel (so
 * kernel_radius plays no part).  Same parameters, discretisation,
 * aggregation and feature ids as mapping, plus id 101 (FR_SCALAR_STDDEV),
 * the statistic of Table 2's scalar column that has no map.  Counts are exact integers; the
 * features are computed in FP64 (MCC in FP32).
 *
 * fr_scalar_plan: discretisation plan and whole-VOI count buffers (about
 *   8 B per volume voxel + 12 B per VOI voxel + 13 x Ng x max(nx, ny, nz) x 4
 *   B); synchronous; mask as for fr_map_plan.  Errors as fr_map_plan.
 * fr_scalar_run: image_dev int16 [nz][ny][nx] on the plan's device; out_dev
 *   double [n_features] (selected features in id order), caller-owned, on the
 *   device.  Asynchronous on s; one run at a time per plan.  Device errors
 *   (Ng > 255 for FBW) are reported by fr_scalar_sync_status, and the outputs
 *   are then NaN.  Results are bit-identical between runs: the GLSZM cell
 *   sums, which visit a hash table whose slot order depends on thread
 *   timing, are added as exact fixed-point integers. */
typedef struct fr_scalar fr_scalar;
fr_status fr_scalar_plan(const fr_map_params* p, const uint8_t* mask, fr_scalar** out);
fr_status fr_scalar_run(fr_scalar* sp, const int16_t* image_dev, double* out_dev,
                        fr_stream_t s);
fr_status fr_scalar_sync_status(fr_scalar* sp);
fr_status fr_scalar_query(const fr_scalar* sp, int64_t* n_voi, int32_t* n_features,
                          size_t* device_bytes);
void fr_scalar_destroy(fr_scalar* sp);

/* Continuous-batching server (iteration-level scheduling).  Requests are
 * planned as they arrive (fr_server_add: synchronous, allocates the request's
 * device state; mask, image and out are device pointers that must stay valid
 * until the request is released).  Each fr_server_step launches the mapping
 * kernel once over up to `voxel_budget` voxels taken round-robin from every
 * request with work left, so a request added while others are being mapped
 * joins the next step and shares its launches with them.  Steps run in order
 * on the server's own stream, at most two in flight (a third waits for the
 * oldest).  fr_server_poll reports finished requests (their maps are
 * complete in `out`) with their status; fr_server_release frees a finished
 * request's device memory and slot.  max_radius bounds the requests' kernel
 * radius (it sizes the launch); max_slots bounds the requests held at once.
 * A server is driven from one host thread. */
typedef struct fr_server fr_server;
fr_status fr_server_create(int32_t device, int32_t max_radius, int32_t max_slots,
                           const fr_tune* tune, fr_server** out);
fr_status fr_server_add(fr_server* s, const fr_map_params* p, const uint8_t* mask,
                        const int16_t* image, float* out, int64_t* id);
fr_status fr_server_step(fr_server* s, int64_t voxel_budget, int32_t* n_active);
fr_status fr_server_poll(fr_server* s, int32_t wait, int64_t* done_ids, int32_t* done_status,
                         int32_t cap, int32_t* n_done);
fr_status fr_server_release(fr_server* s, int64_t id);
fr_status fr_server_query(const fr_server* s, int32_t* active, int32_t* inflight_steps,
                          size_t* device_bytes);
void fr_server_destroy(fr_server* s);

/* Measured issue throughput of the 32-bit ALU pipes of `device` (a
 * measurement helper for the roofline of the mapping kernel, which is bound
 * by plain integer / logic / fp32 instruction issue; the paper has no
 * counterpart).  Every thread of a full-occupancy grid runs 8 dependency
 * chains of one operation: int32 adds, int32 multiply-adds, fp32 fused
 * multiply-adds; the best of 3 timed launches (CUDA events) of each gives
 * lane operations per second, one instruction counted as one operation.
 * Takes about 100 ms; allocates 64 bytes.  Errors: INVALID_ARG (NULL
 * outputs), UNSUPPORTED, CUDA. */
fr_status fr_measure_alu_peak(int32_t device, double* int32_add_per_s, double* int32_mad_per_s,
                              double* fp32_fma_per_s);

/* Allocation-free VOI voxel list.  The paper has no counterpart: this is a
 * service for callers that cannot allocate device memory -- callers whose
 * device memory already belongs to another allocator (a framework's caching
 * pool, an application arena reserved at start-up) or that must not allocate
 * while they run.  It writes into voi (device pointer, int32, room for
 * `capacity` entries) the linear index (z*ny + y)*nx + x of every nonzero
 * voxel of mask (device pointer, uint8 [nz][ny][nx]) in increasing order --
 * the output column order of every map -- and their count into *n_voi (host).
 * It calls no cudaMalloc, cudaFree or other allocating routine: its only
 * scratch is a fixed 2 MiB static device array (per-row counts and offsets)
 * that every GPU loading the library holds until the process exits.
 *   Limits: ny * nz <= FR_NOALLOC_MAX_ROWS and nx * ny * nz < 2^31, else
 *   FR_ERR_UNSUPPORTED.  If the list does not fit in `capacity`, *n_voi still
 *   receives the count, voi is left untouched and FR_ERR_INVALID_ARG returns.
 *   `device` becomes the calling thread's current device.  The first call on
 *   a device looks up the scratch's device address (once per device, with
 *   that device current): make that first call before any stream capture.
 *   The address is kept for the life of the process: after a
 *   cudaDeviceReset of that device it is stale, so the entry point must not
 *   be used again in that process.  An error left pending by earlier CUDA
 *   work of the thread is returned (and cleared) as FR_ERR_CUDA before
 *   anything is launched.
 *   Every call shares the scratch and overwrites every word of it that it
 *   reads; calls that overlap on the GPU (other streams, other threads) race.
 *   The call synchronises stream s once, to read the count; the list itself
 *   is then written asynchronously on s. */
enum { FR_NOALLOC_MAX_ROWS = 262144 };
fr_status fr_voxel_list_noalloc(const uint8_t* mask, int32_t nx, int32_t ny, int32_t nz,
                                int32_t* voi, int64_t capacity, int64_t* n_voi,
                                int32_t device, fr_stream_t s);

/* ---- HDF5 drain of finished results (host only; the paper's "Structured
 * HDF5 storage": one file per extraction with the results, the image and
 * mask arrays, the voxel geometry, the extraction settings and the input's
 * identification; scalar results as ordered feature names and float64
 * values, spatial results as named maps; LZF or gzip compression).
 *
 * File layout (HDF5, superblock version 0, readable by any HDF5 reader):
 *   /image     int16 [nz][ny][nx]   chunked, compressed
 *   /mask      uint8 [nz][ny][nx]   chunked, compressed
 *   /maps/<feature name>   float32 [nz][ny][nx], NaN outside the VOI, one
 *              per selected feature (spatial files); attribute feature_id.
 *              Chunks holding no VOI voxel are not stored (fill value NaN).
 *   /features/names  fixed-length strings [n], /features/values float64 [n]
 *              in feature-id order (scalar files)
 *   root attributes: format, mode ("spatial" / "scalar"), shape_zyx,
 *   spacing_xyz_mm, origin_xyz_mm, discretisation, bin_count, bin_width,
 *   fbw_anchor, kernel_radius, glcm_distance, aggregation, kurtosis_excess,
 *   feature_ids, source, created_utc, writer.
 * Chunks are encoded on host threads; gzip needs the system zlib (libz.so.1,
 * loaded at first use; without it gzip returns FR_ERR_UNSUPPORTED).  The
 * chunk grid holds at most 64 chunks (requested extents grow until it does).
 * Errors: INVALID_ARG (NULL pointer, bad option, row count not matching the
 * selection, voxel index outside the volume), UNSUPPORTED, OOM, IO (the file
 * could not be created or written; a partial file may remain). */
enum { FR_H5_NONE = 0, FR_H5_GZIP = 1, FR_H5_LZF = 2 };

typedef struct fr_h5_options {
  int32_t codec;    /* FR_H5_NONE, FR_H5_GZIP (default) or FR_H5_LZF            */
  int32_t level;    /* gzip level 1..9 (0: 4)                                   */
  int32_t shuffle;  /* 1: HDF5 byte-shuffle filter before the codec (default)   */
  int32_t threads;  /* host threads encoding chunks (0: all hardware threads)   */
  int32_t chunk[3]; /* chunk extents z, y, x (0: a quarter of the extent)       */
} fr_h5_options;

/* The extraction's input, all host memory owned by the caller. */
typedef struct fr_h5_source {
  const int16_t* image;  /* [nz][ny][nx]                                        */
  const uint8_t* mask;   /* [nz][ny][nx], nonzero = VOI                         */
  double origin[3];      /* position of voxel (0,0,0) in mm, x y z              */
  const char* source_id; /* identifies the input (path, UID ...); may be NULL   */
} fr_h5_source;

/* Defaults: gzip level 4 with shuffle, all threads, automatic chunks. */
fr_status fr_h5_options_init(fr_h5_options* o);

/* Spatial extraction: maps (host float32 [n_rows][n_voi], the fr_map_run
 * output for p's selection) with voxel_index (host int32 [n_voi], the
 * linear index z-major of each column, as fr_plan_voxel_index gives).
 * n_rows must equal the number of features p selects.  opt may be NULL. */
fr_status fr_h5_write_maps(const char* path, const fr_map_params* p, const fr_h5_source* src,
                           const float* maps, int32_t n_rows, int64_t n_voi,
                           const int32_t* voxel_index, const fr_h5_options* opt);

/* Scalar extraction: values (host float64 [n_values], the fr_scalar_run
 * output for p's selection, feature-id order).  opt may be NULL. */
fr_status fr_h5_write_scalar(const char* path, const fr_map_params* p, const fr_h5_source* src,
                             const double* values, int32_t n_values, const fr_h5_options* opt);

/* Names and helpers. */
int32_t fr_feature_count(void);        /* map features: FR_NUM_FEATURES */
int32_t fr_scalar_feature_count(void); /* scalar features: FR_NUM_SCALAR_FEATURES */
const char* fr_feature_name(int32_t id); /* NULL outside 0..101 (101: scalar only) */
const char* fr_status_string(fr_status s);
/* Direction i (0..12) as (dz, dy, dx); INVALID_ARG outside 0..12. */
fr_status fr_direction(int32_t i, int32_t* dz, int32_t* dy, int32_t* dx);

#ifdef __cplusplus
}
#endif
#endif /* FLASHMAP_H */
