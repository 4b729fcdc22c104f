// Host-side binned-SAH BVH builder, blob serialiser/validator and the
// Poisson-disc point generator used by the scene generators.
//
// The paper only states that queries run over "a BVH built over some
// primitives" (Section 3.1) traversed with the while-while scheme (Section
// 3.2); construction is not described.  This file produces that structure as
// plain data (boxes and a permutation).  It contains no ray arithmetic and is
// shared by every consumer of a blob purely as an input producer.
//
// Blob format: see include/vsr_bvh.h.

#include "vsr_bvh.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <string>
#include <thread>
#include <vector>

namespace {

thread_local std::string g_bvh_err;

int bvh_fail(const std::string& msg) {
    g_bvh_err = msg;
    return -1;
}

constexpr float kInf = std::numeric_limits<float>::infinity();
constexpr uint32_t kMedianDepth = 40;  // below this depth SAH, then median

struct Box {
    float lo[3] = {kInf, kInf, kInf};
    float hi[3] = {-kInf, -kInf, -kInf};
    void grow(const float* l, const float* h) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], l[a]);
            hi[a] = std::max(hi[a], h[a]);
        }
    }
    void grow_point(const float* p) { grow(p, p); }
    bool empty() const { return lo[0] > hi[0]; }
    double half_area() const {
        if (empty()) return 0.0;
        double dx = (double)hi[0] - lo[0], dy = (double)hi[1] - lo[1],
               dz = (double)hi[2] - lo[2];
        return dx * dy + dy * dz + dz * dx;
    }
};

struct Ref {
    float lo[3], hi[3], c[3];
    uint32_t prim;
};

struct Task {
    uint32_t node, begin, end, depth;
};

uint64_t fnv1a64(const uint8_t* p, size_t n) {
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

struct Header {
    char magic[8];
    uint32_t version, header_bytes, num_nodes, num_prims, max_depth, leaf_max,
        num_leaves, flags;
    uint64_t payload_bytes, checksum, reserved;
};
static_assert(sizeof(Header) == 64, "blob header must be 64 bytes");
static_assert(sizeof(vsr_bvh_node) == 32, "node must be 32 bytes");

class Builder {
   public:
    Builder(std::vector<Ref>&& refs, const vsr_build_params& p)
        : refs_(std::move(refs)), p_(p) {}

    // Build the whole tree.  The top of the tree is built serially until a
    // subtree holds at most `defer` references; those subtrees are built on
    // threads, each into its own node array over its own (disjoint) range of
    // references, and appended in creation order.  The result does not depend
    // on the number of threads or their timing.
    void run() {
        nodes_.reserve(refs_.size() * 2 + 2);
        nodes_.resize(2);
        std::memset(nodes_.data(), 0, sizeof(vsr_bvh_node) * 2);
        if (refs_.empty()) return;
        const uint32_t n = (uint32_t)refs_.size();
        const uint32_t defer = std::max<uint32_t>(n / 256u, 4096u);
        std::vector<Task> deferred;
        process({{0, 0, n, 0}}, nodes_, max_depth_, num_leaves_, defer, &deferred);
        if (deferred.empty()) return;
        struct Sub {
            std::vector<vsr_bvh_node> nodes;
            uint32_t depth = 0, leaves = 0;
        };
        std::vector<Sub> subs(deferred.size());
        std::atomic<size_t> next{0};
        auto worker = [&]() {
            for (size_t k = next++; k < deferred.size(); k = next++) {
                const Task& t = deferred[k];
                Sub& sb = subs[k];
                sb.nodes.resize(1);
                std::memset(sb.nodes.data(), 0, sizeof(vsr_bvh_node));
                process({{0, t.begin, t.end, t.depth}}, sb.nodes, sb.depth, sb.leaves, 0u,
                        nullptr);
            }
        };
        unsigned nt = std::thread::hardware_concurrency();
        if (const char* e = std::getenv("VSR_BUILD_THREADS")) nt = (unsigned)std::atoi(e);
        nt = std::max(1u, std::min<unsigned>(nt, (unsigned)deferred.size()));
        std::vector<std::thread> pool;
        for (unsigned k = 1; k < nt; ++k) pool.emplace_back(worker);
        worker();
        for (auto& th : pool) th.join();
        for (size_t k = 0; k < deferred.size(); ++k) {
            Sub& sb = subs[k];
            const uint32_t base = (uint32_t)nodes_.size();  // even: pairs only
            auto remap = [&](vsr_bvh_node nd) {
                if ((nd.count_axis >> 2) == 0) nd.left_or_first = base + nd.left_or_first - 1u;
                return nd;
            };
            nodes_[deferred[k].node] = remap(sb.nodes[0]);
            for (size_t j = 1; j < sb.nodes.size(); ++j) nodes_.push_back(remap(sb.nodes[j]));
            max_depth_ = std::max(max_depth_, sb.depth);
            num_leaves_ += sb.leaves;
        }
    }

    // Binned-SAH construction of the subtrees on `stack` into `nodes`.  A
    // task whose node is nodes[t.node] covers refs_[t.begin, t.end); child
    // pairs are appended to `nodes`.  With `deferred`, tasks of at most
    // `defer` references (and more than a leaf) are set aside instead.
    void process(std::vector<Task> stack, std::vector<vsr_bvh_node>& nodes, uint32_t& max_depth,
                 uint32_t& leaves, uint32_t defer, std::vector<Task>* deferred) {
        std::vector<uint32_t> cnt(p_.bins);
        std::vector<Box> bbox(p_.bins);
        std::vector<double> right_area(p_.bins);
        std::vector<uint32_t> right_cnt(p_.bins);
        while (!stack.empty()) {
            Task t = stack.back();
            stack.pop_back();
            if (deferred && t.end - t.begin <= defer && t.end - t.begin > p_.leaf_max) {
                deferred->push_back(t);
                continue;
            }
            Box nb, cb;
            for (uint32_t i = t.begin; i < t.end; ++i) {
                nb.grow(refs_[i].lo, refs_[i].hi);
                cb.grow_point(refs_[i].c);
            }
            vsr_bvh_node& nd = nodes[t.node];
            for (int a = 0; a < 3; ++a) {
                nd.lo[a] = nb.lo[a];
                nd.hi[a] = nb.hi[a];
            }
            const uint32_t n = t.end - t.begin;
            max_depth = std::max(max_depth, t.depth);
            if (n == 1) {
                make_leaf(t, nodes, leaves);
                continue;
            }
            int axis = -1;
            uint32_t mid = t.begin;
            bool sah_ok = false;
            if (t.depth < kMedianDepth) {
                // Binned SAH over the three axes.
                double best = std::numeric_limits<double>::infinity();
                int best_axis = -1;
                uint32_t best_split = 0;
                for (int a = 0; a < 3; ++a) {
                    const float ext = cb.hi[a] - cb.lo[a];
                    if (!(ext > 0.0f)) continue;
                    const float scale = (float)p_.bins / ext;
                    std::fill(cnt.begin(), cnt.end(), 0u);
                    std::fill(bbox.begin(), bbox.end(), Box());
                    for (uint32_t i = t.begin; i < t.end; ++i) {
                        uint32_t k = bin_of(refs_[i].c[a], cb.lo[a], scale);
                        cnt[k]++;
                        bbox[k].grow(refs_[i].lo, refs_[i].hi);
                    }
                    Box acc;
                    uint32_t ac = 0;
                    for (int k = (int)p_.bins - 1; k > 0; --k) {
                        acc.grow(bbox[k].lo, bbox[k].hi);
                        ac += cnt[k];
                        right_area[k] = acc.half_area();
                        right_cnt[k] = ac;
                    }
                    Box lacc;
                    uint32_t lc = 0;
                    for (uint32_t k = 1; k < p_.bins; ++k) {
                        lacc.grow(bbox[k - 1].lo, bbox[k - 1].hi);
                        lc += cnt[k - 1];
                        if (lc == 0 || right_cnt[k] == 0) continue;
                        double c = lacc.half_area() * lc + right_area[k] * right_cnt[k];
                        if (c < best) {
                            best = c;
                            best_axis = a;
                            best_split = k;
                        }
                    }
                }
                if (best_axis >= 0) {
                    const double na = nb.half_area();
                    const double split_cost =
                        p_.traversal_cost + (na > 0.0 ? best / na : (double)n);
                    if (n <= p_.leaf_max && (double)n <= split_cost) {
                        make_leaf(t, nodes, leaves);
                        continue;
                    }
                    const int a = best_axis;
                    const float ext = cb.hi[a] - cb.lo[a];
                    const float scale = (float)p_.bins / ext;
                    const float clo = cb.lo[a];
                    const uint32_t bins = p_.bins;
                    auto it = std::partition(
                        refs_.begin() + t.begin, refs_.begin() + t.end,
                        [&](const Ref& r) {
                            return bin_of_n(r.c[a], clo, scale, bins) < best_split;
                        });
                    mid = (uint32_t)(it - refs_.begin());
                    axis = a;
                    sah_ok = mid > t.begin && mid < t.end;
                }
            }
            if (!sah_ok) {
                if (n <= p_.leaf_max) {
                    make_leaf(t, nodes, leaves);
                    continue;
                }
                // Object median along the widest centroid axis (index split
                // when all centroids coincide).
                int a = 0;
                float ext = cb.hi[0] - cb.lo[0];
                for (int k = 1; k < 3; ++k)
                    if (cb.hi[k] - cb.lo[k] > ext) {
                        ext = cb.hi[k] - cb.lo[k];
                        a = k;
                    }
                mid = t.begin + n / 2;
                if (ext > 0.0f) {
                    std::nth_element(refs_.begin() + t.begin, refs_.begin() + mid,
                                     refs_.begin() + t.end,
                                     [a](const Ref& x, const Ref& y) {
                                         if (x.c[a] != y.c[a]) return x.c[a] < y.c[a];
                                         return x.prim < y.prim;
                                     });
                }
                axis = a;
            }
            const uint32_t left = (uint32_t)nodes.size();
            nodes.resize(nodes.size() + 2);
            vsr_bvh_node& nd2 = nodes[t.node];  // resize may move storage
            nd2.left_or_first = left;
            nd2.count_axis = (uint32_t)axis;
            stack.push_back({left + 1, mid, t.end, t.depth + 1});
            stack.push_back({left, t.begin, mid, t.depth + 1});
        }
    }

    int serialise(void** blob, size_t* bytes) const {
        const uint64_t payload = 32ull * nodes_.size() + 4ull * refs_.size();
        const size_t total = 64 + (size_t)payload;
        uint8_t* out = (uint8_t*)std::malloc(total);
        if (!out) return bvh_fail("vsr_bvh_build: out of host memory");
        Header h;
        std::memset(&h, 0, sizeof(h));
        std::memcpy(h.magic, VSR_BVH_MAGIC, 8);
        h.version = VSR_BVH_VERSION;
        h.header_bytes = VSR_BVH_HEADER_BYTES;
        h.num_nodes = (uint32_t)nodes_.size();
        h.num_prims = (uint32_t)refs_.size();
        h.max_depth = max_depth_;
        h.leaf_max = p_.leaf_max;
        h.num_leaves = num_leaves_;
        h.payload_bytes = payload;
        uint8_t* pay = out + 64;
        std::memcpy(pay, nodes_.data(), 32ull * nodes_.size());
        uint32_t* order = (uint32_t*)(pay + 32ull * nodes_.size());
        for (size_t i = 0; i < refs_.size(); ++i) order[i] = refs_[i].prim;
        h.checksum = fnv1a64(pay, (size_t)payload);
        std::memcpy(out, &h, 64);
        *blob = out;
        *bytes = total;
        return 0;
    }

    uint32_t max_depth() const { return max_depth_; }

   private:
    static uint32_t bin_of_n(float c, float lo, float scale, uint32_t bins) {
        float f = (c - lo) * scale;
        int k = (int)f;
        if (k < 0) k = 0;
        if (k >= (int)bins) k = (int)bins - 1;
        return (uint32_t)k;
    }
    uint32_t bin_of(float c, float lo, float scale) const {
        return bin_of_n(c, lo, scale, p_.bins);
    }
    static void make_leaf(const Task& t, std::vector<vsr_bvh_node>& nodes, uint32_t& leaves) {
        vsr_bvh_node& nd = nodes[t.node];
        nd.left_or_first = t.begin;
        nd.count_axis = (t.end - t.begin) << 2;
        ++leaves;
    }

    std::vector<Ref> refs_;
    vsr_build_params p_;
    std::vector<vsr_bvh_node> nodes_;
    uint32_t max_depth_ = 0;
    uint32_t num_leaves_ = 0;
};

// SplitMix64 (Steele, Lea, Flood 2014) for the Poisson-disc sampler.
struct SplitMix64 {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

}  // namespace

extern "C" {

const char* vsr_bvh_last_error(void) { return g_bvh_err.c_str(); }

void vsr_bvh_free(void* blob) { std::free(blob); }

int vsr_bvh_build(const float* verts, uint64_t nverts, const uint32_t* idx,
                  uint32_t ntri, const vsr_build_params* params, void** blob,
                  size_t* bytes) {
    g_bvh_err.clear();
    if (!blob || !bytes) return bvh_fail("vsr_bvh_build: null output pointer");
    *blob = nullptr;
    *bytes = 0;
    if (ntri > 0 && !verts) return bvh_fail("vsr_bvh_build: null verts");
    if (ntri > (1u << 28)) return bvh_fail("vsr_bvh_build: more than 2^28 triangles");
    vsr_build_params p{4u, 32u, 1.0f};
    if (params) p = *params;
    if (p.leaf_max < 1 || p.leaf_max > VSR_BVH_MAX_LEAF)
        return bvh_fail("vsr_bvh_build: leaf_max must be in 1..8");
    if (p.bins < 4 || p.bins > 256) return bvh_fail("vsr_bvh_build: bins must be in 4..256");
    if (!(p.traversal_cost >= 0.0f) || !std::isfinite(p.traversal_cost))
        return bvh_fail("vsr_bvh_build: traversal_cost must be finite and >= 0");
    if (idx == nullptr && nverts < 3ull * ntri)
        return bvh_fail("vsr_bvh_build: non-indexed layout needs 3*ntri vertices");
    std::vector<Ref> refs(ntri);
    for (uint32_t i = 0; i < ntri; ++i) {
        Ref& r = refs[i];
        for (int a = 0; a < 3; ++a) {
            r.lo[a] = kInf;
            r.hi[a] = -kInf;
        }
        for (int k = 0; k < 3; ++k) {
            uint64_t vi = idx ? (uint64_t)idx[3ull * i + k] : 3ull * i + k;
            if (vi >= nverts) return bvh_fail("vsr_bvh_build: vertex index out of range");
            const float* v = verts + 3 * vi;
            for (int a = 0; a < 3; ++a) {
                if (!std::isfinite(v[a]))
                    return bvh_fail("vsr_bvh_build: non-finite vertex coordinate");
                r.lo[a] = std::min(r.lo[a], v[a]);
                r.hi[a] = std::max(r.hi[a], v[a]);
            }
        }
        for (int a = 0; a < 3; ++a) r.c[a] = 0.5f * r.lo[a] + 0.5f * r.hi[a];
        r.prim = i;
    }
    Builder b(std::move(refs), p);
    b.run();
    if (b.max_depth() > VSR_BVH_MAX_DEPTH)
        return bvh_fail("vsr_bvh_build: depth limit exceeded");
    return b.serialise(blob, bytes);
}

int vsr_bvh_build_boxes(const float* boxes, uint32_t n, const vsr_build_params* params,
                        void** blob, size_t* bytes) {
    g_bvh_err.clear();
    if (!blob || !bytes) return bvh_fail("vsr_bvh_build_boxes: null output pointer");
    *blob = nullptr;
    *bytes = 0;
    if (n > 0 && !boxes) return bvh_fail("vsr_bvh_build_boxes: null boxes");
    if (n > (1u << 28)) return bvh_fail("vsr_bvh_build_boxes: more than 2^28 boxes");
    vsr_build_params p{4u, 32u, 1.0f};
    if (params) p = *params;
    if (p.leaf_max < 1 || p.leaf_max > VSR_BVH_MAX_LEAF)
        return bvh_fail("vsr_bvh_build_boxes: leaf_max must be in 1..8");
    if (p.bins < 4 || p.bins > 256) return bvh_fail("vsr_bvh_build_boxes: bins must be in 4..256");
    if (!(p.traversal_cost >= 0.0f) || !std::isfinite(p.traversal_cost))
        return bvh_fail("vsr_bvh_build_boxes: traversal_cost must be finite and >= 0");
    std::vector<Ref> refs(n);
    for (uint32_t i = 0; i < n; ++i) {
        Ref& r = refs[i];
        for (int a = 0; a < 3; ++a) {
            r.lo[a] = boxes[6ull * i + a];
            r.hi[a] = boxes[6ull * i + 3 + a];
            if (!std::isfinite(r.lo[a]) || !std::isfinite(r.hi[a]) || r.lo[a] > r.hi[a])
                return bvh_fail("vsr_bvh_build_boxes: box " + std::to_string(i) +
                                " is not finite with lo <= hi");
            r.c[a] = 0.5f * r.lo[a] + 0.5f * r.hi[a];
        }
        r.prim = i;
    }
    Builder b(std::move(refs), p);
    b.run();
    if (b.max_depth() > VSR_BVH_MAX_DEPTH)
        return bvh_fail("vsr_bvh_build_boxes: depth limit exceeded");
    return b.serialise(blob, bytes);
}

int vsr_bvh_validate(const void* blob, size_t bytes) {
    g_bvh_err.clear();
    if (!blob) return bvh_fail("blob: null pointer");
    if (bytes < 64) return bvh_fail("blob: shorter than the 64-byte header");
    Header h;
    std::memcpy(&h, blob, 64);
    if (std::memcmp(h.magic, VSR_BVH_MAGIC, 8) != 0) return bvh_fail("blob: bad magic");
    if (h.version != VSR_BVH_VERSION) return bvh_fail("blob: unsupported version");
    if (h.header_bytes != VSR_BVH_HEADER_BYTES) return bvh_fail("blob: bad header size");
    if (h.num_nodes < 2) return bvh_fail("blob: fewer than 2 nodes");
    if (h.num_prims > (1u << 28)) return bvh_fail("blob: too many primitives");
    const uint64_t payload = 32ull * h.num_nodes + 4ull * h.num_prims;
    if (h.payload_bytes != payload) return bvh_fail("blob: payload size mismatch");
    if (bytes != 64 + payload) return bvh_fail("blob: truncated or oversized");
    const uint8_t* pay = (const uint8_t*)blob + 64;
    if (fnv1a64(pay, (size_t)payload) != h.checksum) return bvh_fail("blob: checksum mismatch");
    if (h.max_depth > VSR_BVH_MAX_DEPTH) return bvh_fail("blob: max_depth above 64");
    if (h.leaf_max < 1 || h.leaf_max > VSR_BVH_MAX_LEAF) return bvh_fail("blob: bad leaf_max");
    std::vector<vsr_bvh_node> nodes(h.num_nodes);
    std::memcpy(nodes.data(), pay, 32ull * h.num_nodes);
    std::vector<uint32_t> order(h.num_prims);
    std::memcpy(order.data(), pay + 32ull * h.num_nodes, 4ull * h.num_prims);
    if (h.num_prims == 0) {
        if (h.num_nodes != 2) return bvh_fail("blob: empty BVH must have 2 nodes");
        return 0;
    }
    std::vector<uint8_t> seen_node(h.num_nodes, 0), seen_slot(h.num_prims, 0),
        seen_prim(h.num_prims, 0);
    struct Item {
        uint32_t node, depth;
    };
    std::vector<Item> st;
    st.push_back({0, 0});
    seen_node[0] = 1;
    uint32_t leaves = 0, deepest = 0;
    while (!st.empty()) {
        Item it = st.back();
        st.pop_back();
        const vsr_bvh_node& nd = nodes[it.node];
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(nd.lo[a]) || !std::isfinite(nd.hi[a]) || nd.lo[a] > nd.hi[a])
                return bvh_fail("blob: invalid node bounds");
        if (it.depth > h.max_depth) return bvh_fail("blob: node deeper than max_depth");
        deepest = std::max(deepest, it.depth);
        const uint32_t count = nd.count_axis >> 2, axis = nd.count_axis & 3u;
        if (count == 0) {
            const uint32_t l = nd.left_or_first;
            if (axis > 2) return bvh_fail("blob: bad split axis");
            if (l < 2 || (l & 1u) || (uint64_t)l + 1 >= h.num_nodes)
                return bvh_fail("blob: child index out of range");
            // descent then strictly increases the node index, which bounds
            // every traversal loop without a per-step counter
            if (l <= it.node) return bvh_fail("blob: children must follow their parent");
            for (uint32_t c = l; c <= l + 1; ++c) {
                if (seen_node[c]) return bvh_fail("blob: node reached twice");
                seen_node[c] = 1;
                const vsr_bvh_node& ch = nodes[c];
                for (int a = 0; a < 3; ++a)
                    if (ch.lo[a] < nd.lo[a] || ch.hi[a] > nd.hi[a])
                        return bvh_fail("blob: child box not inside parent box");
                st.push_back({c, it.depth + 1});
            }
        } else {
            if (count > h.leaf_max) return bvh_fail("blob: leaf larger than leaf_max");
            const uint64_t f = nd.left_or_first;
            if (f + count > h.num_prims) return bvh_fail("blob: leaf range out of range");
            for (uint64_t s = f; s < f + count; ++s) {
                if (seen_slot[s]) return bvh_fail("blob: primitive slot in two leaves");
                seen_slot[s] = 1;
                const uint32_t pr = order[s];
                if (pr >= h.num_prims) return bvh_fail("blob: primitive id out of range");
                if (seen_prim[pr]) return bvh_fail("blob: primitive listed twice");
                seen_prim[pr] = 1;
            }
            ++leaves;
        }
    }
    for (uint32_t s = 0; s < h.num_prims; ++s)
        if (!seen_slot[s]) return bvh_fail("blob: primitive slot not covered by a leaf");
    for (uint32_t i = 2; i < h.num_nodes; ++i)
        if (!seen_node[i]) return bvh_fail("blob: unreachable node");
    if (leaves != h.num_leaves) return bvh_fail("blob: leaf count mismatch");
    if (deepest != h.max_depth) return bvh_fail("blob: max_depth mismatch");
    return 0;
}

int vsr_inputs_poisson_disc(float w, float h, float r, uint32_t max_points,
                            uint64_t seed, float* out_xy, uint32_t* out_n) {
    g_bvh_err.clear();
    if (!out_xy || !out_n) return bvh_fail("poisson: null output");
    if (!(w > 0) || !(h > 0) || !(r > 0)) return bvh_fail("poisson: bad extents");
    const double cell = r / std::sqrt(2.0);
    const int64_t gw = (int64_t)std::ceil(w / cell), gh = (int64_t)std::ceil(h / cell);
    if (gw * gh > (int64_t)1 << 31) return bvh_fail("poisson: grid too large");
    std::vector<int32_t> grid((size_t)(gw * gh), -1);
    std::vector<float> pts;
    std::vector<int32_t> active;
    SplitMix64 rng{seed};
    const double r2 = (double)r * r;
    auto insert = [&](double x, double y) {
        int32_t id = (int32_t)(pts.size() / 2);
        pts.push_back((float)x);
        pts.push_back((float)y);
        int64_t gx = (int64_t)(x / cell), gy = (int64_t)(y / cell);
        grid[(size_t)(gy * gw + gx)] = id;
        active.push_back(id);
    };
    insert(rng.uniform() * w, rng.uniform() * h);
    while (!active.empty()) {
        size_t ai = (size_t)(rng.next() % active.size());
        int32_t id = active[ai];
        const double px = pts[2 * id], py = pts[2 * id + 1];
        bool placed = false;
        for (int k = 0; k < 30 && !placed; ++k) {
            const double ang = 6.283185307179586 * rng.uniform();
            const double rad = std::sqrt(r2 + 3.0 * r2 * rng.uniform());
            const double x = px + rad * std::cos(ang), y = py + rad * std::sin(ang);
            if (x < 0 || y < 0 || x >= w || y >= h) continue;
            const int64_t gx = (int64_t)(x / cell), gy = (int64_t)(y / cell);
            if (gx >= gw || gy >= gh) continue;
            bool ok = true;
            for (int64_t yy = std::max<int64_t>(0, gy - 2); ok && yy <= std::min(gh - 1, gy + 2); ++yy)
                for (int64_t xx = std::max<int64_t>(0, gx - 2); xx <= std::min(gw - 1, gx + 2); ++xx) {
                    int32_t q = grid[(size_t)(yy * gw + xx)];
                    if (q < 0) continue;
                    const double dx = pts[2 * q] - x, dy = pts[2 * q + 1] - y;
                    if (dx * dx + dy * dy < r2) {
                        ok = false;
                        break;
                    }
                }
            if (ok) {
                insert(x, y);
                placed = true;
            }
        }
        if (!placed) {
            active[ai] = active.back();
            active.pop_back();
        }
    }
    const uint32_t total = (uint32_t)(pts.size() / 2);
    std::vector<uint32_t> pick(total);
    for (uint32_t i = 0; i < total; ++i) pick[i] = i;
    const uint32_t n = std::min(total, max_points);
    for (uint32_t i = 0; i < n; ++i) {  // partial Fisher-Yates
        uint32_t j = i + (uint32_t)(rng.next() % (uint64_t)(total - i));
        std::swap(pick[i], pick[j]);
    }
    std::sort(pick.begin(), pick.begin() + n);
    for (uint32_t i = 0; i < n; ++i) {
        out_xy[2 * i] = pts[2 * pick[i]];
        out_xy[2 * i + 1] = pts[2 * pick[i] + 1];
    }
    *out_n = n;
    return 0;
}

}  // extern "C"
