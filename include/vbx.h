/* vbx.h -- C ABI of the GB300 (sm_103a) per-scan map update of Voxblox
 * (Oleynikova et al., arXiv 1611.03631): grouped-raycast TSDF fusion into a block-hashed
 * map, the incremental ESDF update from the changed TSDF voxels, trilinear
 * distance/gradient queries, and the incremental mesh of the TSDF iso-surface.
 *
 * Conventions for every entry point:
 *  - All pointers named *_dev are device pointers (CUDA global memory) owned by the caller;
 *    all other pointers are host pointers owned by the caller. The library keeps no pointer
 *    to caller memory after the work it enqueued has finished.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream). Work is
 *    enqueued on it in order; calls that return host data synchronise that stream.
 *  - The map owns its device memory (block hash, voxel pools, frontiers, per-scan scratch).
 *  - Every call returns a vbx_status. Errors detected on the device (hash probe limit,
 *    block pool exhausted, a device loop exceeding its round or wait budget) are recorded
 *    in a sticky per-map error word and reported by the next call that synchronises
 *    (vbx_sync, vbx_get_stats, the export calls). After VBX_ERR_HASH_FULL or
 *    VBX_ERR_OUT_OF_MEMORY the map stays usable; voxels of blocks that could not be
 *    allocated are not integrated.
 *  - vbx_last_error() returns a thread-local message for the last non-OK status.
 *  - Voxel coordinates are integer triples i with voxel centre (i + 1/2) * voxel_size.
 *    Block (bx,by,bz) holds voxels [b*B, b*B + B) per axis; inside a block the local index
 *    of voxel (lx,ly,lz) is (lz*B + ly)*B + lx.
 */
#ifndef VBX_H_
#define VBX_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vbx_map_s* vbx_map_t;

typedef enum {
  VBX_OK = 0,
  VBX_ERR_INVALID_ARG = 1,   /* bad size, pointer or parameter; nothing was enqueued */
  VBX_ERR_OUT_OF_MEMORY = 2, /* device allocation failed or the block pool is exhausted */
  VBX_ERR_HASH_FULL = 3,     /* block hash probe limit reached */
  VBX_ERR_TIMEOUT = 4,       /* a device loop exceeded its round budget or a wait its limit
                                (grid barriers, the ESDF work queue)                         */
  VBX_ERR_CUDA = 5,          /* a CUDA runtime call failed (message in vbx_last_error) */
  VBX_ERR_CAPACITY = 6       /* an output buffer is too small: the sizes needed are reported
                                and the map is unchanged                                     */
} vbx_status;

/* Map options (Sec. IV-A weighting, Sec. IV-B merging, Sec. V-A fixed band). */
typedef struct {
  int weighting;          /* 0: constant weight, Eq. (2); 1: 1/z^2 with linear drop-off
                             behind the surface, Eq. (4)                                    */
  float eps;              /* drop-off start epsilon of Eq. (4); <= 0 selects voxel_size     */
  float fixed_band;       /* gamma, ESDF fixed band |D| < gamma (Sec. V-A); <= 0 selects
                             voxel_size (the one-voxel band recommended in Sec. VI-B)       */
  float w_max;            /* W_max of Eq. (3); <= 0 selects 1e4 (the paper gives no value)  */
  float max_range;        /* points farther than this from the sensor are dropped;
                             <= 0 or +inf: no limit                                          */
  int grouped;            /* 1: grouped raycasting, one ray per voxel holding points
                             (Sec. IV-B); 0: one ray per point                              */
  int64_t block_capacity; /* blocks in the voxel pool (device memory budget); 0: 2^25/B^3  */
  int64_t max_points;     /* initial per-scan point capacity; grows on demand; 0: 1<<20     */
  int64_t scratch_blocks; /* blocks one scan may enter (each holds the scan's per-voxel sums,
                             33 B per voxel); 0 or more than block_capacity: block_capacity.
                             A scan that enters more blocks is not integrated at all and its
                             synchronising call reports VBX_ERR_OUT_OF_MEMORY               */
  int esdf_mode;          /* ESDF seeds: 0 the fixed band |D| < fixed_band (Sec. V-A); 1 the
                             occupancy ESDF compared in Sec. VI-B: observed voxels with D < 0
                             are occupied at distance 0 and every other observed voxel holds
                             its unsigned distance to them                                   */
  int euclidean;          /* 0: quasi-Euclidean distances (26-neighbour steps v, v*sqrt(2),
                             v*sqrt(3), the parent is a neighbour direction); 1: full Euclidean
                             distances, each voxel keeping the offset to its site, the fixed
                             voxel it is measured to (Sec. V-A, Sec. VI-B). Requires
                             max_esdf_dist / voxel_size <= 126. Such maps are updated one at a
                             time (vbx_update_esdf), not in batches. The result depends on the
                             processing order: every voxel's distance is exactly what its site
                             offers it, |d_site| + v * |offset|, the site is an observed fixed
                             voxel of its sign, and no observed same-sign neighbour's site
                             offers it less                                                  */
} vbx_map_options;

/* Fills *opt with the defaults above (weighting 0, grouped 1). */
vbx_status vbx_default_options(vbx_map_options* opt);

/* Creates a map of voxel size v (> 0, metres), blocks of voxels_per_block^3 voxels
 * (4, 8 or 16), truncation distance delta (>= v) and ESDF maximum distance d_max (> 0).
 * Sec. III: layers of fixed-size blocks indexed by block position through a hash table.
 * opt may be NULL (defaults). On success *out holds the new map. Allocates device memory
 * on the current device: about 26 bytes per pool voxel, 33 bytes per scratch voxel
 * (scratch_blocks x B^3) and the per-scan point buffers (vbx_map_bytes gives the total). */
vbx_status vbx_create_map(float voxel_size, int voxels_per_block, float truncation, float max_esdf_dist,
                          const vbx_map_options* opt, vbx_map_t* out);

/* Frees all device memory of the map (synchronises the device). NULL is accepted. */
vbx_status vbx_destroy_map(vbx_map_t map);

/* Integrates one posed scan into the TSDF (Sec. IV: Eq. (1)-(4), grouped raycasting).
 * points_dev: n x 3 float32, row-major, sensor frame; non-finite rows are dropped.
 * T_world_sensor: 16 float32, row-major 4x4 homogeneous pose (host memory, copied).
 * Rays run from the sensor origin to truncation distance behind each (grouped) point; each
 * traversed voxel receives the projective distance of Eq. (1), truncated, with the weight of
 * Eq. (2) or (4); all of a scan's updates of one voxel are merged by Eq. (3) at once.
 * Updated voxels are queued for the next vbx_update_esdf. n = 0 is a no-op. */
vbx_status vbx_integrate_scan(vbx_map_t map, const float* points_dev, int64_t n, const float T_world_sensor[16],
                              void* stream);

/* vbx_integrate_scan for callers that must not allocate device memory while they run, such
 * as a robot's real-time loop (cudaMalloc/cudaFree synchronise the whole device and can stall
 * it past the loop's deadline) or a process that committed its device-memory budget at
 * start-up. The paper has no counterpart: it only changes where the per-scan scratch lives.
 * Same arguments and results as vbx_integrate_scan, but the scratch (point group table, group
 * list, ray buffer) is a file-scope device array of the library sized for at most 65536
 * points; n above 65536 returns VBX_ERR_INVALID_ARG and enqueues nothing. The call allocates
 * nothing. Every GPU that loads the library holds that array (about 9.3 MiB) until exit. The
 * first call on a device looks up the array's device address (cudaGetSymbolAddress); make that
 * first call before any stream capture. All calls share the array: calls whose work overlaps
 * on the GPU (other streams, other maps at the same time) race and must be serialised. The
 * current device must be the map's device. */
vbx_status vbx_integrate_scan_noalloc(vbx_map_t map, const float* points_dev, int64_t n, const float T_world_sensor[16],
                                      void* stream);

/* Updates the ESDF incrementally from the TSDF voxels updated since the last call
 * (Sec. V-A, Algorithm 1): fixed band |D| < gamma, raise wavefront, then lower wavefront over
 * 26-connected neighbours with quasi-Euclidean steps v, v*sqrt(2), v*sqrt(3), capped at
 * d_max. Runs as one cooperative persistent kernel on `stream`. A CTA stages an active tile
 * (a block, or an 8^3 octant of a 16^3 block) with its one-voxel halo in shared memory and
 * relaxes it to local convergence. For one map each wave runs as a work queue of tiles; batches
 * with more than 16 maps at work run each wave in global rounds. Both give the same ESDF. */
vbx_status vbx_update_esdf(vbx_map_t map, void* stream);

/* Distance and gradient queries (the planner's interface, Sec. VII; trilinear interpolation
 * as in Sec. VI-A). q_dev: n x 3 float32 world points. Outputs (device, caller-owned):
 * dist_dev n float32, grad_dev n x 3 float32, status_dev n uint8 (0 = ok, 1 = unknown: one of
 * the 8 surrounding voxel centres is unobserved; dist/grad are NaN then). */
vbx_status vbx_query_distance_gradient(vbx_map_t map, const float* q_dev, int64_t n, float* dist_dev,
                                       float* grad_dev, uint8_t* status_dev, void* stream);

/* Waits for `stream` and returns (and clears) the map's sticky device error, if any. */
vbx_status vbx_sync(vbx_map_t map, void* stream);

typedef struct {
  int64_t points_in;      /* points passed to the last vbx_integrate_scan                  */
  int64_t points_valid;   /* of those, accepted by the filter                               */
  int64_t rays;           /* rays cast (groups when grouped, else valid points)             */
  int64_t records;        /* voxel updates with w > 0 emitted by the rays                  */
  int64_t updated;        /* distinct voxels updated by the last scan                       */
  int64_t new_blocks;     /* blocks allocated by the last scan                              */
  int64_t blocks;         /* blocks in the map                                              */
  int64_t esdf_in;        /* TSDF voxels consumed by the last vbx_update_esdf               */
  int64_t seeds;          /* of those, in the fixed band                                    */
  int64_t raise_pops;     /* voxels processed by the raise wave                             */
  int64_t lower_pops;     /* voxels processed by the lower wave                             */
  int64_t raise_rounds;   /* global rounds of the raise wave; 1 when it ran as one work
                             queue (16 or fewer maps with work in the launch), 0 if empty  */
  int64_t lower_rounds;   /* the same for the lower wave                                    */
  int64_t launches;       /* kernels launched by this map since creation                    */
  int64_t esdf_block_visits; /* tiles staged in shared memory by the last ESDF update        */
  int64_t esdf_local_iters;  /* local relaxation iterations summed over those stagings       */
  int64_t esdf_classify_ns;  /* device time of the classification phase of the last update  */
  int64_t esdf_raise_ns;     /* ... of the raise wave                                         */
  int64_t esdf_lower_ns;     /* ... of the lower wave                                         */
  int64_t touched_blocks;    /* blocks the rays of the last scan entered (scratch blocks it
                                needed; above scratch_blocks the scan was rejected)          */
} vbx_stats;

/* Synchronises `stream`, then fills *out. Returns the sticky device error if one is set. */
vbx_status vbx_get_stats(vbx_map_t map, vbx_stats* out, void* stream);

/* Number of blocks in the map (synchronises `stream`). */
vbx_status vbx_num_blocks(vbx_map_t map, int64_t* n_out, void* stream);

/* Copies the map to host memory in pool order (block allocation order), cap >= number of
 * blocks (else VBX_ERR_INVALID_ARG). Any output pointer may be NULL to skip it.
 *   keys:   cap x 3 int32 block coordinates
 *   tsdf:   cap x B^3 x 2 float32 (D, W) per voxel
 *   esdf_d: cap x B^3 float32 ESDF distance per voxel
 *   parent: cap x B^3 uint8, direction to the parent voxel (k = (dx+1)*9+(dy+1)*3+(dz+1), 255 none);
 *           Euclidean maps: the low byte of the word (use vbx_export_sites)
 *   flags:  cap x B^3 uint8, bit0 observed, bit1 fixed, bit2 holds a site (Euclidean maps)
 * Synchronises `stream`. */
vbx_status vbx_export_blocks(vbx_map_t map, int32_t* keys, float* tsdf, float* esdf_d, uint8_t* parent,
                             uint8_t* flags, int64_t cap, void* stream);

/* Euclidean maps (options.euclidean = 1): the site of every voxel, in the block order of
 * vbx_export_blocks. offsets: cap x B^3 x 3 int8 (site - voxel, in voxels), has_site: cap x B^3
 * (1: the voxel holds a site; fixed voxels are their own sites and report 0). Host buffers,
 * either may be NULL. Synchronising; VBX_ERR_INVALID_ARG for a quasi-Euclidean map. */
vbx_status vbx_export_sites(vbx_map_t map, int8_t* offsets, uint8_t* has_site, int64_t cap, void* stream);

/* Voxel coordinates (cap x 3 int32, host) of the voxels updated by the last
 * vbx_integrate_scan or vbx_import_tsdf, in unspecified order; *n_out = their number
 * (entries beyond cap are not written). Synchronises `stream`. */
vbx_status vbx_export_updated(vbx_map_t map, int32_t* vox, int64_t cap, int64_t* n_out, void* stream);

/* Sets TSDF voxels directly (host arrays: vox n x 3 int32, D n float32, W n float32), allocating
 * their blocks, and queues them for the next vbx_update_esdf exactly as if a scan had updated
 * them. Used to restore a saved map and to drive the ESDF from given TSDF values.
 * Duplicate voxels in one call are not allowed. Synchronises `stream`. */
vbx_status vbx_import_tsdf(vbx_map_t map, const int32_t* vox, const float* D, const float* W, int64_t n,
                           void* stream);

/* One block of an extracted mesh: its key (the block holds voxels key*B .. key*B + B - 1 on
   each axis), the number of triangles of the cells whose minimum corner it holds, and the
   index of the first of them in the triangle arrays (a block's triangles are contiguous). */
typedef struct {
  int32_t key[3];
  uint32_t num_triangles;
  int64_t first_triangle;
} vbx_mesh_block;

/* Iso-surface D = 0 of the TSDF as triangles: the mesh layer that Sec. III builds from updated
   TSDF voxels on demand (marching cubes, Sec. II; the paper fixes no variant, so this is the
   rule below).
   A cell is the cube between 8 neighbouring voxel centres, ((float)index + 0.5f) * voxel_size;
   it is meshed when all 8 voxels are observed (W > 0) and belongs to the block holding its
   minimum corner. A corner is inside when D < 0 (so -0 and +0 are outside). Every cube edge
   whose ends differ carries the vertex pa + t (pb - pa), t = Da / (Da - Db), each float32
   operation rounded to nearest. On each face the crossings are joined so that the inside
   corners lie to the left of the boundary walked counter-clockwise seen from outside; a face
   with four crossings cuts off each inside corner alone. The joined segments form loops (each
   started at its lowest-numbered edge: edges 0-3 along x, 4-7 along y, 8-11 along z, corner
   c = x + 2y + 4z); a loop of 3 vertices is one triangle, a loop of k > 3 the k triangles
   (centroid, vertex i+1, vertex i) around the float32 mean of its vertices. Triangles are wound
   so that (b - a) x (c - a) points to positive D. The surface is closed wherever it stays
   inside observed space, and neighbouring cells share its edges with opposite directions.
   updated_only = 0 meshes every block. updated_only = 1 meshes only the blocks whose mesh may
   have changed since the last successful call: those with a cell that has a voxel in a block
   that a scan's rays entered or vbx_import_tsdf wrote since then. A caller that keeps the
   meshes per block replaces the listed blocks' meshes with the returned ones (a listed block
   with no triangles has none). vbx_reset_map clears every mark.
   Outputs, device memory, blocks in any order:
     cells_dev  int32 [tri_cap][4], 16-byte aligned: the cell's minimum-corner voxel (x, y, z)
                and the triangle's index within the cell;
     verts_dev  float32 [tri_cap][3][3]: vertices a, b, c in world coordinates;
     blocks_dev vbx_mesh_block [block_cap].
   *n_tri_out and *n_blocks_out receive the sizes needed. If either exceeds its capacity the
   call returns VBX_ERR_CAPACITY, the outputs are incomplete and no mark is cleared, so a call
   with larger buffers returns the same set. Synchronises the stream. */
vbx_status vbx_extract_mesh(vbx_map_t map, int updated_only, int32_t* cells_dev, float* verts_dev, int64_t tri_cap,
                            vbx_mesh_block* blocks_dev, int64_t block_cap, int64_t* n_tri_out, int64_t* n_blocks_out,
                            void* stream);

/* Per-kernel timing with CUDA events recorded on the launch stream around each kernel of
 * this map (off by default). */
vbx_status vbx_set_profiling(vbx_map_t map, int enable);

/* Names (static strings) and accumulated milliseconds / launch counts of the profiled
 * kernels; *n_out = number of kernel kinds (<= cap written). Synchronises `stream`.
 * vbx_reset_kernel_times clears the accumulators. */
vbx_status vbx_get_kernel_times(vbx_map_t map, const char** names, double* ms, int64_t* launches, int cap,
                                int* n_out, void* stream);
vbx_status vbx_reset_kernel_times(vbx_map_t map);

/* ---- Batched form: many independent maps advanced by the same launches --------------------
 * A batch has a fixed number of slots, each bound to one map (all on the current device, no map
 * in two slots). One step integrates one scan per slot, updates every slot's ESDF in one
 * cooperative launch and answers every slot's distance/gradient queries, with about seven
 * kernel launches in total whatever the number of slots; with VBX_STEP_GRAPH the step is
 * captured once into a CUDA graph per flag set and replayed. Each map's results are the same
 * as when it is updated alone (the per-map arithmetic does not depend on the batch). The paper
 * has no batched form; it is how many robots' maps share one GPU. */
typedef struct vbx_batch_s* vbx_batch_t;

typedef struct {
  const float* points_dev;  /* n x 3 float32, sensor frame (device, caller-owned) */
  int64_t n;                /* 0: no scan for this slot in this step */
  float T_world_sensor[16]; /* row-major 4x4 pose */
} vbx_scan_in;

typedef struct {
  const float* q_dev;   /* n x 3 float32 world points (device) */
  int64_t n;            /* 0: no queries for this slot */
  float* dist_dev;      /* n float32 (device) */
  float* grad_dev;      /* n x 3 float32 (device) */
  uint8_t* status_dev;  /* n uint8 (device), as vbx_query_distance_gradient */
} vbx_query_io;

enum { VBX_STEP_INTEGRATE = 1, VBX_STEP_ESDF = 2, VBX_STEP_QUERY = 4, VBX_STEP_GRAPH = 8 };

/* Creates a batch of `count` slots (1..256) bound to maps[0..count). max_queries bounds the
 * query count per slot and step. A slot's scan may hold at most as many points as its map's
 * per-scan capacity (vbx_map_options.max_points rounded up to a power of two, or the largest
 * scan the map has integrated alone); batches never grow a map's scratch. */
vbx_status vbx_batch_create(const vbx_map_t* maps, int count, int64_t max_queries, vbx_batch_t* out);

/* Rebinds slot `slot` to `map` (same device, not bound to another slot). Steps already issued keep
 * the map they were issued with; the next step takes the new one. The call synchronises the
 * device only when the map needs larger ESDF work lists or a larger block edge than the batch has
 * held so far (it reallocates them, at least doubling the lists), so binding maps of the kinds
 * already bound never stalls steps in flight. */
vbx_status vbx_batch_bind(vbx_batch_t batch, int slot, vbx_map_t map);

/* One batched step on `stream`: scans[count] (VBX_STEP_INTEGRATE), ESDF update of every slot
 * (VBX_STEP_ESDF), queries[count] (VBX_STEP_QUERY, may be NULL otherwise). Host arrays are copied
 * before the call returns. The staged descriptors form a ring of 4: the call waits for the step
 * issued four calls earlier, so up to 4 steps may be in flight on the stream. */
vbx_status vbx_batch_step(vbx_batch_t batch, const vbx_scan_in* scans, const vbx_query_io* queries, int flags,
                          void* stream);

/* Chooses launch shapes (CTAs per SM of the traversal kernel; threads per CTA and CTAs per SM of
 * the ESDF kernel) by timing full steps on the given inputs: one untimed step, then the better of
 * two steps per candidate; a candidate replaces the current best only when it is more than 3 %
 * faster. The scans ARE integrated into the maps at every step, so call it on warm-up data. Writes a one-line description to report (may be NULL) that ends with
 * "trial_steps=<number of steps it ran>". */
vbx_status vbx_batch_autotune(vbx_batch_t batch, const vbx_scan_in* scans, const vbx_query_io* queries, int flags,
                              void* stream, char* report, int report_len);

/* Per-kernel CUDA-event timing of this batch's direct (non-graph) steps, as vbx_set_profiling and
 * vbx_get_kernel_times do for a map. */
vbx_status vbx_batch_set_profiling(vbx_batch_t batch, int enable);
vbx_status vbx_batch_kernel_times(vbx_batch_t batch, const char** names, double* ms, int64_t* launches, int cap,
                                  int* n_out, void* stream);

/* Waits for `stream`; returns the first sticky device error of the bound maps (and clears it). */
vbx_status vbx_batch_sync(vbx_batch_t batch, void* stream);

vbx_status vbx_batch_destroy(vbx_batch_t batch);

/* Device bytes a map created with these parameters allocates (pool, hash, lists, per-scan
 * scratch for opt->max_points points), for admission control against a memory budget. */
vbx_status vbx_map_bytes(int voxels_per_block, const vbx_map_options* opt, int64_t* bytes_out);

/* Device bytes the map holds now. */
vbx_status vbx_map_device_bytes(vbx_map_t map, int64_t* bytes_out);

/* Empties the map (no blocks, no observed voxels, nothing queued) without freeing its memory,
 * so that it can serve a new session. Enqueued on `stream` (one kernel and one memset, sized on
 * the device by the map's own counters); the host does not wait. Work enqueued on the same
 * stream afterwards sees the empty map. */
vbx_status vbx_reset_map(vbx_map_t map, void* stream);

/* Kernels launched by all maps of this process (a running counter). */
int64_t vbx_total_launches(void);

/* Thread-local message describing the last error returned on this thread ("" if none). */
const char* vbx_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* VBX_H_ */
