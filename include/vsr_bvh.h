/*
 * vsr_bvh.h — host-side BVH construction and the serialised BVH blob format.
 *
 * The paper's queries run over a BVH of primitives (Section 3.1), traversed
 * with Aila and Laine's while-while scheme (Section 3.2), but it does not say
 * how the BVH is built.  This library builds it once on the host with a binned
 * surface-area heuristic and serialises it into a self-describing blob.  The
 * blob is plain data: the GPU loader (vsr_bvh_load in vsr.h) and any other
 * consumer parse it on their own.  The builder computes only bounding boxes and
 * a primitive permutation; it performs no ray arithmetic.
 *
 * Blob layout (little endian, all fields naturally aligned):
 *
 *   offset  size  field
 *   0       8     magic          "VSRBVH01"
 *   8       4     version        1
 *   12      4     header_bytes   64
 *   16      4     num_nodes      >= 2 (node 1 is padding so that sibling
 *                                pairs start at even indices)
 *   20      4     num_prims      number of triangles referenced (== scene ntri)
 *   24      4     max_depth      edges on the longest root-to-leaf path (<= 64)
 *   28      4     leaf_max       largest leaf primitive count (1..8)
 *   32      4     num_leaves
 *   36      4     flags          0
 *   40      8     payload_bytes  32*num_nodes + 4*num_prims
 *   48      8     checksum       FNV-1a 64 over the payload bytes
 *   56      8     reserved       0
 *   64      ...   nodes[num_nodes]     (vsr_bvh_node, 32 B each)
 *   ...           prim_order[num_prims] (uint32, original triangle ids in
 *                                        leaf order)
 *
 * Node semantics: node 0 is the root.  count = count_axis >> 2,
 * axis = count_axis & 3.  count == 0: inner node whose children are the two
 * adjacent nodes left_or_first (even, >= 2, and above the node's own index:
 * children follow their parent) and left_or_first + 1, split along `axis`
 * (0, 1, 2).  count > 0: leaf holding prim_order[left_or_first ..
 * left_or_first + count).  Every triangle appears in exactly one leaf.  A blob
 * with num_prims == 0 has num_nodes == 2, an all-zero root and is traced as
 * "every ray misses".
 */
#ifndef VSR_BVH_H
#define VSR_BVH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VSR_BVH_MAGIC "VSRBVH01"
#define VSR_BVH_VERSION 1u
#define VSR_BVH_HEADER_BYTES 64u
#define VSR_BVH_MAX_DEPTH 64u
#define VSR_BVH_MAX_LEAF 8u

typedef struct vsr_bvh_node {
    float lo[3];
    uint32_t left_or_first;
    float hi[3];
    uint32_t count_axis;
} vsr_bvh_node;

typedef struct vsr_build_params {
    uint32_t leaf_max;   /* 1..8, default 4 */
    uint32_t bins;       /* SAH bins per axis, 4..256, default 32 */
    float traversal_cost; /* SAH cost of one inner node relative to one
                             triangle test, default 1.0 */
} vsr_build_params;

/*
 * Build a binned-SAH BVH over indexed triangles and serialise it.
 *   verts  host, float32 [nverts*3], xyz per vertex
 *   idx    host, uint32 [ntri*3], vertex indices per triangle; NULL means the
 *          non-indexed layout verts[(3*i + k)*3 ..] for corner k of triangle i
 *   params NULL selects the defaults above
 *   blob   receives a buffer allocated by this library (free with
 *          vsr_bvh_free); bytes receives its size.
 * Returns 0 on success, a negative value on invalid arguments (null pointers,
 * out-of-range indices, non-finite vertices, bad params) or allocation
 * failure; vsr_bvh_last_error() then describes the problem.
 * Ownership: the caller keeps verts/idx; the blob belongs to the caller.
 */
int vsr_bvh_build(const float* verts, uint64_t nverts, const uint32_t* idx,
                  uint32_t ntri, const vsr_build_params* params, void** blob,
                  size_t* bytes);

/*
 * The same builder over axis-aligned boxes (the primitives of a top-level
 * BVH whose leaves hold instances, each a BVH of its own; Section 3.2 on
 * BVHs acting as compound primitives).  Primitive i of the blob is box i.
 *   boxes  host, float32 [n*6]: lo.xyz, hi.xyz per box, finite, lo <= hi
 * Returns and ownership as vsr_bvh_build.
 */
int vsr_bvh_build_boxes(const float* boxes, uint32_t n, const vsr_build_params* params,
                        void** blob, size_t* bytes);

/* Release a blob returned by vsr_bvh_build or vsr_bvh_build_boxes. NULL is
 * ignored. */
void vsr_bvh_free(void* blob);

/* Structural validation of a blob (magic, version, sizes, checksum, child and
 * primitive index ranges, depth, permutation).  0 when valid, negative
 * otherwise with vsr_bvh_last_error() set. */
int vsr_bvh_validate(const void* blob, size_t bytes);

/* Message of the last failure on the calling thread ("" if none). */
const char* vsr_bvh_last_error(void);

/*
 * Seeded Poisson-disc point set over [0,w) x [0,h) with minimum distance r
 * (Bridson's algorithm run until the active list empties, then a seeded
 * random subset of max_points).  out_xy: host float32 [max_points*2];
 * *out_n receives the number written (<= max_points).  Used by the scene
 * generators; it is not part of the traversal.
 */
int vsr_inputs_poisson_disc(float w, float h, float r, uint32_t max_points,
                            uint64_t seed, float* out_xy, uint32_t* out_n);

#ifdef __cplusplus
}
#endif

#endif /* VSR_BVH_H */
