// Octree of Section 3.7: the domain is scaled to a cube, refined uniformly to depth l_max,
// empty boxes are skipped, boxes are found by bit interleaving (Morton keys) and sorting, and
// the near-field (27-box neighbourhood) and M2L interaction lists are built.
//
// Everything runs on the device: bounding-cube reduction, 30-bit Morton keys, a stable LSD
// radix sort written here (8-bit digits, per-warp match ranking), per-level unique boxes by
// flag + scan, parents and neighbours by binary search over the sorted box keys.
#include "internal.h"

#include <algorithm>
#include <cmath>

namespace bem {

// ------------------------------------------------------------------------------ scratch
namespace {
struct Scratch {
    DevBuf<int32_t> a, b, c;
};
Scratch &scan_scratch(int depth) {
    static Scratch s[4];
    return s[depth];
}

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Exclusive scan of one tile per block; writes the tile total to sums[block].
__global__ void k_scan_tiles(const int32_t *__restrict__ in, int32_t *__restrict__ out, int64_t n,
                             int32_t *__restrict__ sums) {
    __shared__ int32_t warp_tot[SCAN_THREADS / 32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int32_t v[SCAN_ITEMS];
    int32_t t = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        t += v[i];
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t incl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        int32_t x = lane < SCAN_THREADS / 32 ? warp_tot[lane] : 0;
        int32_t xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += y;
        }
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = xi - x;
        if (lane == SCAN_THREADS / 32 - 1 && sums) sums[blockIdx.x] = xi;
    }
    __syncthreads();
    int32_t run = warp_tot[w] + incl - t;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

__global__ void k_scan_add(int32_t *__restrict__ out, int64_t n, const int32_t *__restrict__ offs) {
    int64_t i = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x;
    int32_t o = offs[blockIdx.x];
    for (int k = 0; k < SCAN_ITEMS; ++k, i += SCAN_THREADS)
        if (i < n) out[i] += o;
}

__global__ void k_scan_total(const int32_t *in, const int32_t *ex, int64_t n, int32_t *total) {
    *total = (n > 0) ? ex[n - 1] + in[n - 1] : 0;
}

void scan_rec(const int32_t *in, int32_t *out, int64_t n, cudaStream_t st, int depth) {
    int nb = div_up(n, SCAN_TILE);
    if (nb <= 1) {
        k_scan_tiles<<<1, SCAN_THREADS, 0, st>>>(in, out, n, nullptr);
        BEM_LAUNCH_CHECK();
        return;
    }
    if (depth >= 3) fail(BEM_ERR_ARG, "scan too large");
    Scratch &s = scan_scratch(depth);
    s.a.resize(nb);
    s.b.resize(nb);
    k_scan_tiles<<<nb, SCAN_THREADS, 0, st>>>(in, out, n, s.a.p);
    BEM_LAUNCH_CHECK();
    scan_rec(s.a.p, s.b.p, nb, st, depth + 1);
    k_scan_add<<<nb, SCAN_THREADS, 0, st>>>(out, n, s.b.p);
    BEM_LAUNCH_CHECK();
}
}  // namespace

void exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *total_dev, cudaStream_t st) {
    if (n <= 0) return;
    scan_rec(in, out, n, st, 0);
    if (total_dev) {
        k_scan_total<<<1, 1, 0, st>>>(in, out, n, total_dev);
        BEM_LAUNCH_CHECK();
    }
}

// ------------------------------------------------------------------------------ radix sort
namespace {
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_WARPS = RS_THREADS / 32;

__global__ void k_rs_hist(const uint32_t *__restrict__ keys, int64_t n, int shift,
                          int32_t *__restrict__ hist, int nblocks) {
    __shared__ int32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; ++r) {
        int64_t i = base + r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: items keep their input order within a digit. Items are taken in rounds of
// RS_THREADS consecutive keys; a warp ranks equal digits with __match_any_sync and warps are
// ordered through a shared per-digit prefix.
__global__ void k_rs_scatter(const uint32_t *__restrict__ kin, const int32_t *__restrict__ vin,
                             uint32_t *__restrict__ kout, int32_t *__restrict__ vout, int64_t n,
                             int shift, const int32_t *__restrict__ offs, int nblocks) {
    __shared__ int32_t running[256];
    __shared__ int32_t total[256];
    __shared__ int32_t wcnt[RS_WARPS][256];
    int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    running[tid] = offs[(int64_t)tid * nblocks + blockIdx.x];
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; ++r) {
        for (int k = 0; k < 8; ++k) wcnt[w][lane * 8 + k] = 0;
        int64_t i = base + r * RS_THREADS + tid;
        bool valid = i < n;
        uint32_t key = valid ? kin[i] : 0u;
        int32_t val = valid ? vin[i] : 0;
        int d = valid ? (int)((key >> shift) & 255u) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & ((1u << lane) - 1u));
        __syncwarp();
        if (valid && rank == 0) wcnt[w][d] = __popc(peers);
        __syncthreads();
        {
            int acc = 0;
            for (int ww = 0; ww < RS_WARPS; ++ww) {
                int t = wcnt[ww][tid];
                wcnt[ww][tid] = acc;
                acc += t;
            }
            total[tid] = acc;
        }
        __syncthreads();
        if (valid) {
            int pos = running[d] + wcnt[w][d] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        running[tid] += total[tid];
        __syncthreads();
    }
}
}  // namespace

// Sort (keys, vals) by the low `bits` bits of the keys, stably. Result ends in keys/vals.
void radix_sort_u32(uint32_t *keys, int32_t *vals, int64_t n, int bits, uint32_t *keys_tmp,
                    int32_t *vals_tmp, cudaStream_t st) {
    if (n <= 1) return;
    int nblocks = div_up(n, RS_TILE);
    static DevBuf<int32_t> hist, offs;
    hist.resize((size_t)256 * nblocks);
    offs.resize((size_t)256 * nblocks);
    uint32_t *ka = keys, *kb = keys_tmp;
    int32_t *va = vals, *vb = vals_tmp;
    int passes = 0;
    for (int shift = 0; shift < bits; shift += 8) {
        k_rs_hist<<<nblocks, RS_THREADS, 0, st>>>(ka, n, shift, hist.p, nblocks);
        BEM_LAUNCH_CHECK();
        exclusive_scan_i32(hist.p, offs.p, (int64_t)256 * nblocks, nullptr, st);
        k_rs_scatter<<<nblocks, RS_THREADS, 0, st>>>(ka, va, kb, vb, n, shift, offs.p, nblocks);
        BEM_LAUNCH_CHECK();
        std::swap(ka, kb);
        std::swap(va, vb);
        ++passes;
    }
    if (passes & 1) {
        BEM_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
        BEM_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    }
}

// ------------------------------------------------------------------------------ Morton helpers
namespace {
__device__ __forceinline__ uint32_t spread3(uint32_t x) {
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}
__device__ __forceinline__ uint32_t compact3(uint32_t x) {
    x &= 0x09249249u;
    x = (x ^ (x >> 2)) & 0x030C30C3u;
    x = (x ^ (x >> 4)) & 0x0300F00Fu;
    x = (x ^ (x >> 8)) & 0xFF0000FFu;
    x = (x ^ (x >> 16)) & 0x000003FFu;
    return x;
}
__device__ __forceinline__ uint32_t morton(uint32_t gx, uint32_t gy, uint32_t gz) {
    return (spread3(gx) << 2) | (spread3(gy) << 1) | spread3(gz);
}
__device__ __forceinline__ void demorton(uint32_t k, int &gx, int &gy, int &gz) {
    gx = (int)compact3(k >> 2);
    gy = (int)compact3(k >> 1);
    gz = (int)compact3(k);
}
// Index of the first element >= key in the sorted array a[0..n).
__device__ __forceinline__ int lower_bound_u32(const uint32_t *a, int n, uint32_t key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ int find_box(const uint32_t *a, int n, uint32_t key) {
    int i = lower_bound_u32(a, n, key);
    return (i < n && a[i] == key) ? i : -1;
}

__global__ void k_bbox(int64_t N, const double *__restrict__ xyz, double *__restrict__ part) {
    // part[block][6] = min x,y,z, max x,y,z
    __shared__ double sm[6][256];
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        for (int d = 0; d < 3; ++d) {
            double v = xyz[d * N + i];
            mn[d] = fmin(mn[d], v);
            mx[d] = fmax(mx[d], v);
        }
    }
    for (int d = 0; d < 3; ++d) {
        sm[d][threadIdx.x] = mn[d];
        sm[3 + d][threadIdx.x] = mx[d];
    }
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int d = 0; d < 3; ++d) {
                sm[d][threadIdx.x] = fmin(sm[d][threadIdx.x], sm[d][threadIdx.x + s]);
                sm[3 + d][threadIdx.x] = fmax(sm[3 + d][threadIdx.x], sm[3 + d][threadIdx.x + s]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) part[blockIdx.x * 6 + threadIdx.x] = sm[threadIdx.x][0];
}

__global__ void k_keys(int64_t N, const double *__restrict__ xyz, double ox, double oy, double oz,
                       double inv_size, uint32_t *__restrict__ key, int32_t *__restrict__ idx) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double scale = inv_size * (double)(1 << kDeepLevel);
    int g[3];
    double o[3] = {ox, oy, oz};
    for (int d = 0; d < 3; ++d) {
        double u = (xyz[d * N + i] - o[d]) * scale;
        int gi = (int)floor(u);
        g[d] = min(max(gi, 0), (1 << kDeepLevel) - 1);
    }
    key[i] = morton(g[0], g[1], g[2]);
    idx[i] = (int32_t)i;
}

// Clusters: the key is (cluster << 24) | 24-bit Morton key of depth 8 in the cluster's own cube,
// so sorting groups clusters and shifting right by 3 (8 - l) gives (cluster << 3l) | box key.
constexpr int kClusterDeep = 8;

__global__ void k_cluster_bbox(const int64_t *__restrict__ cvoff, int64_t N, const double *__restrict__ xyz,
                               double *__restrict__ out) {
    __shared__ double sm[6][256];
    const int c = blockIdx.x;
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = cvoff[c] + threadIdx.x; i < cvoff[c + 1]; i += blockDim.x)
        for (int d = 0; d < 3; ++d) {
            double v = xyz[d * N + i];
            mn[d] = fmin(mn[d], v);
            mx[d] = fmax(mx[d], v);
        }
    for (int d = 0; d < 3; ++d) {
        sm[d][threadIdx.x] = mn[d];
        sm[3 + d][threadIdx.x] = mx[d];
    }
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int d = 0; d < 3; ++d) {
                sm[d][threadIdx.x] = fmin(sm[d][threadIdx.x], sm[d][threadIdx.x + s]);
                sm[3 + d][threadIdx.x] = fmax(sm[3 + d][threadIdx.x], sm[3 + d][threadIdx.x + s]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) out[c * 6 + threadIdx.x] = sm[threadIdx.x][0];
}

// cube[c] = (origin x, y, z, 1 / size)
__global__ void k_keys_clusters(int64_t N, const double *__restrict__ xyz, const int32_t *__restrict__ vcid,
                                const double *__restrict__ cube, uint32_t *__restrict__ key, int32_t *__restrict__ idx) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int c = vcid[i];
    const double scale = cube[4 * c + 3] * (double)(1 << kClusterDeep);
    int g[3];
    for (int d = 0; d < 3; ++d) {
        double u = (xyz[d * N + i] - cube[4 * c + d]) * scale;
        int gi = (int)floor(u);
        g[d] = min(max(gi, 0), (1 << kClusterDeep) - 1);
    }
    key[i] = ((uint32_t)c << (3 * kClusterDeep)) | morton(g[0], g[1], g[2]);
    idx[i] = (int32_t)i;
}

// unique[l] += number of i in [1, N) where the level-l prefix of the key changes
__global__ void k_level_counts(int64_t N, int deep, const uint32_t *__restrict__ key, int32_t *__restrict__ cnt) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool valid = i >= 1 && i < N;
    uint32_t a = valid ? key[i] : 0u, b = valid ? key[i - 1] : 0u;
    for (int l = 0; l <= deep; ++l) {
        int sh = 3 * (deep - l);
        int f = (valid && (a >> sh) != (b >> sh)) ? 1 : 0;
        int tot = __reduce_add_sync(0xffffffffu, f);
        if ((threadIdx.x & 31) == 0 && tot) atomicAdd(&cnt[l], tot);
    }
}

__global__ void k_flags_points(int64_t N, const uint32_t *__restrict__ key, int shift, int32_t *__restrict__ flag) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    flag[i] = (i == 0 || (key[i] >> shift) != (key[i - 1] >> shift)) ? 1 : 0;
}

// Leaf boxes straight from the sorted points: start, key and the leaf of every point.
__global__ void k_emit_leaves(int64_t N, const uint32_t *__restrict__ key, int shift,
                              const int32_t *__restrict__ flag, const int32_t *__restrict__ ex,
                              uint32_t *__restrict__ bkey, int32_t *__restrict__ bstart,
                              int32_t *__restrict__ leaf_of) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int b = ex[i] + flag[i] - 1;
    leaf_of[i] = b;
    if (flag[i]) {
        bkey[b] = key[i] >> shift;
        bstart[b] = (int32_t)i;
    }
}

__global__ void k_flags_boxes(int n, const uint32_t *__restrict__ ckey, int32_t *__restrict__ flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    flag[i] = (i == 0 || (ckey[i] >> 3) != (ckey[i - 1] >> 3)) ? 1 : 0;
}

// Parents from children (children are sorted, so each parent's children are contiguous).
__global__ void k_emit_parents(int n, const uint32_t *__restrict__ ckey, const int32_t *__restrict__ cstart,
                               const int32_t *__restrict__ flag, const int32_t *__restrict__ ex,
                               uint32_t *__restrict__ pkey, int32_t *__restrict__ pstart,
                               int32_t *__restrict__ cparent, int pbase) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int b = ex[i] + flag[i] - 1;
    cparent[i] = pbase + b;
    if (flag[i]) {
        pkey[b] = ckey[i] >> 3;
        pstart[b] = cstart[i];
    }
}

__global__ void k_box_counts(int n, const int32_t *__restrict__ bstart, int32_t total, int32_t *__restrict__ bcount) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bcount[i] = ((i + 1 < n) ? bstart[i + 1] : total) - bstart[i];
}

// Near field (Section 3.7, A^(sparse)): the non-empty leaves among the 27 around each leaf.
__global__ void k_neighbours(int nleaf, int L, const uint32_t *__restrict__ lkey,
                             const int32_t *__restrict__ lcount, int32_t *__restrict__ nbr,
                             int32_t *__restrict__ ncnt, int8_t *__restrict__ nd,
                             unsigned long long *__restrict__ pairs) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    int gx, gy, gz;
    const uint32_t mask = (1u << (3 * L)) - 1u, pre = lkey[b] & ~mask;  // cluster prefix
    demorton(lkey[b] & mask, gx, gy, gz);
    int lim = 1 << L, c = 0;
    long long src = 0;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
                int x = gx + dx, y = gy + dy, z = gz + dz;
                if (x < 0 || y < 0 || z < 0 || x >= lim || y >= lim || z >= lim) continue;
                int f = find_box(lkey, nleaf, pre | morton(x, y, z));
                if (f < 0) continue;
                nbr[b * 27 + c] = f;
                nd[(b * 27 + c) * 4 + 0] = (int8_t)dx;
                nd[(b * 27 + c) * 4 + 1] = (int8_t)dy;
                nd[(b * 27 + c) * 4 + 2] = (int8_t)dz;
                nd[(b * 27 + c) * 4 + 3] = 0;
                src += lcount[f];
                ++c;
            }
    ncnt[b] = c;
    atomicAdd(pairs, (unsigned long long)(lcount[b] * (src - 1)));
}

// Compact index of an M2L offset (dx,dy,dz) in [-3,3]^3 with max |d| >= 2, in lexicographic
// order; must match the order in which the operator builder enumerates the offsets. It is the
// offset's position among all 343 offsets minus the near offsets (all |d| <= 1) before it.
__device__ __forceinline__ int m2l_class(int dx, int dy, int dz) {
    const int full = (dx + 3) * 49 + (dy + 3) * 7 + (dz + 3);
    auto below = [](int d) { return min(max(d + 1, 0), 3); };  // near values (-1, 0, 1) below d
    const bool nx = dx >= -1 && dx <= 1, ny = dy >= -1 && dy <= 1;
    const int near_before = below(dx) * 9 + (nx ? below(dy) * 3 + (ny ? below(dz) : 0) : 0);
    return full - near_before;
}

// M2L list of a box: children of the parent's neighbours that are not its own neighbours.
// pass 0 counts, pass 1 writes (target, source, class) at `off[b]`.
__global__ void k_m2l_lists(int n, int l, const uint32_t *__restrict__ key, const uint32_t *__restrict__ pkey,
                            int np, int gbase, int pass, int32_t *__restrict__ cnt,
                            const int32_t *__restrict__ off, int32_t *__restrict__ tgt,
                            int32_t *__restrict__ src, uint32_t *__restrict__ cls) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    int gx, gy, gz;
    const uint32_t mask = (1u << (3 * l)) - 1u;
    const uint32_t cl = key[b] >> (3 * l);  // cluster id (0 without clusters)
    const uint32_t pre = cl << (3 * l), ppre = cl << (3 * (l - 1));
    demorton(key[b] & mask, gx, gy, gz);
    int px = gx >> 1, py = gy >> 1, pz = gz >> 1;
    int plim = 1 << (l - 1);
    int c = 0;
    int64_t o = pass ? off[b] : 0;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
                int x = px + dx, y = py + dy, z = pz + dz;
                if (x < 0 || y < 0 || z < 0 || x >= plim || y >= plim || z >= plim) continue;
                const uint32_t pk = ppre | morton(x, y, z);
                if (find_box(pkey, np, pk) < 0) continue;
                // the parent's children are consecutive in key order: key = parent key * 8 + octant
                for (int f = lower_bound_u32(key, n, pk << 3); f < n && (key[f] >> 3) == pk; ++f) {
                    const int oc = (int)(key[f] & 7u);
                    int cx = 2 * x + ((oc >> 2) & 1), cy = 2 * y + ((oc >> 1) & 1), cz = 2 * z + (oc & 1);
                    int ddx = cx - gx, ddy = cy - gy, ddz = cz - gz;
                    if (ddx >= -1 && ddx <= 1 && ddy >= -1 && ddy <= 1 && ddz >= -1 && ddz <= 1) continue;
                    if (pass) {
                        tgt[o + c] = gbase + b;
                        src[o + c] = gbase + f;
                        cls[o + c] = (uint32_t)m2l_class(ddx, ddy, ddz);
                    }
                    ++c;
                }
            }
    if (!pass) cnt[b] = c;
}

__global__ void k_iota(int64_t n, int32_t *a) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) a[i] = (int32_t)i;
}

template <class T>
__global__ void k_gather_i32(int64_t n, const int32_t *__restrict__ idx, const T *__restrict__ in, T *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[idx[i]];
}

__global__ void k_copy_keys(int64_t n, const int32_t *__restrict__ tgt, uint32_t *__restrict__ key,
                            int32_t *__restrict__ cnt) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    key[i] = (uint32_t)tgt[i];
    atomicAdd(&cnt[tgt[i]], 1);
}

__global__ void k_hist_small(int64_t n, const uint32_t *__restrict__ k, int nbins, int32_t *__restrict__ h) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&h[k[i]], 1);
}

// Octant keys of the children at one level, for the child -> parent translation pairs.
__global__ void k_octants(int n, const uint32_t *__restrict__ key, uint32_t *__restrict__ oct, int32_t *__restrict__ id) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    oct[i] = key[i] & 7u;
    id[i] = i;
}

__global__ void k_up_pairs(int n, const int32_t *__restrict__ id, int base, const int32_t *__restrict__ parent,
                           int32_t *__restrict__ child, int32_t *__restrict__ par) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int g = base + id[i];
    child[i] = g;
    par[i] = parent[g];
}

// Sorted-order point data: leaf-local coordinates (units of the leaf box, centred), normals
// and weights.
__global__ void k_sorted_points(int64_t N, int L, int deep, const int32_t *__restrict__ perm,
                                const uint32_t *__restrict__ key, const double *__restrict__ xyz,
                                const double *__restrict__ nrm, const double *__restrict__ s,
                                const double *__restrict__ cube, const int32_t *__restrict__ vcid,
                                double *__restrict__ loc64, float *__restrict__ loc32,
                                double *__restrict__ n64, float *__restrict__ n32,
                                double *__restrict__ s_sorted, double *__restrict__ ih) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int j = perm[i];
    int g[3];
    demorton((key[i] >> (3 * (deep - L))) & ((1u << (3 * L)) - 1u), g[0], g[1], g[2]);
    const int c = vcid ? vcid[j] : 0;
    double o[3] = {cube[4 * c], cube[4 * c + 1], cube[4 * c + 2]};
    double scale = cube[4 * c + 3] * (double)(1 << L);
    ih[i] = scale;
    for (int d = 0; d < 3; ++d) {
        double u = (xyz[d * N + j] - o[d]) * scale - ((double)g[d] + 0.5);
        loc64[d * N + i] = u;
        loc32[d * N + i] = (float)u;
        double nv = nrm[d * N + j];
        n64[d * N + i] = nv;
        n32[d * N + i] = (float)nv;
    }
    s_sorted[i] = s[j];
}
// Near-field work units: leaf b gets ceil(n_b / 64) units (b, 64 u).
__global__ void k_p2p_unit_count(int nleaf, const int32_t *__restrict__ bcount, int32_t *__restrict__ cnt) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nleaf) cnt[b] = (bcount[b] + 63) / 64;
}

__global__ void k_p2p_unit_emit(int nleaf, const int32_t *__restrict__ bcount, const int32_t *__restrict__ off,
                                int2 *__restrict__ units) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    const int n = (bcount[b] + 63) / 64;
    for (int u = 0; u < n; ++u) units[off[b] + u] = make_int2(b, 64 * u);
}

// Symmetric near field: leaf A owns its pairs with the neighbours B > A. S_A = the floats one
// unit of A writes (the points of its owned neighbours, in neighbour-list order); the leaf's
// region holds its units' shares one after another, padded to 32 floats.
__global__ void k_back_sizes(int nleaf, const int32_t *__restrict__ nbr, const int32_t *__restrict__ ncnt,
                             const int32_t *__restrict__ bcount, const int32_t *__restrict__ ucnt,
                             int32_t *__restrict__ S, int32_t *__restrict__ blk32) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nleaf) return;
    int s = 0;
    for (int k = 0; k < ncnt[a]; ++k) {
        const int f = nbr[a * 27 + k];
        if (f > a) s += bcount[f];
    }
    S[a] = s;
    blk32[a] = (int32_t)(((int64_t)ucnt[a] * s + 31) / 32);
}

__global__ void k_back_base(int nleaf, const int32_t *__restrict__ blkoff, int64_t *__restrict__ base) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < nleaf) base[a] = 32 * (int64_t)blkoff[a];
}

// for neighbour k = A of leaf B with A < B: where B's share starts inside each unit of A (the
// owned neighbours of A before B in A's list, summed)
__global__ void k_back_gofs(int nleaf, const int32_t *__restrict__ nbr, const int32_t *__restrict__ ncnt,
                            const int32_t *__restrict__ bcount, int32_t *__restrict__ gofs) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    for (int k = 0; k < 27; ++k) {
        int g = -1;
        if (k < ncnt[b]) {
            const int a = nbr[b * 27 + k];
            if (a < b) {
                int off = 0;
                for (int k2 = 0; k2 < ncnt[a]; ++k2) {
                    const int f = nbr[a * 27 + k2];
                    if (f == b) {
                        g = off;
                        break;
                    }
                    if (f > a) off += bcount[f];
                }
            }
        }
        gofs[b * 27 + k] = g;
    }
}

}  // namespace

// ------------------------------------------------------------------------------ build
void build_tree(Context &c) {
    Tree &t = c.tree;
    cudaStream_t st = c.stream;
    const int64_t N = c.N;
    t.N = N;
    const int tb = 256;

    const bool clusters = c.C > 1;
    t.deep = clusters ? kClusterDeep : kDeepLevel;
    DevBuf<double> &cube = t.s_f64[0];  // per cluster: origin x, y, z, 1 / size
    cube.resize(4 * std::max<int64_t>(c.C, 1));
    std::vector<double> hcube(4 * std::max<int64_t>(c.C, 1));
    // 1. bounding cube (one per cluster)
    int nbb = std::min<int64_t>(div_up(N, tb), 1024);
    DevBuf<double> &part = t.s_f64[1];
    part.resize((size_t)nbb * 6);
    k_bbox<<<nbb, tb, 0, st>>>(N, c.xyz.p, part.p);
    BEM_LAUNCH_CHECK();
    std::vector<double> hp((size_t)nbb * 6);
    BEM_CUDA(cudaMemcpyAsync(hp.data(), part.p, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    BEM_CUDA(cudaStreamSynchronize(st));
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = 0; b < nbb; ++b)
        for (int d = 0; d < 3; ++d) {
            mn[d] = std::min(mn[d], hp[b * 6 + d]);
            mx[d] = std::max(mx[d], hp[b * 6 + 3 + d]);
        }
    double ext = 0.0;
    for (int d = 0; d < 3; ++d) {
        if (!std::isfinite(mn[d]) || !std::isfinite(mx[d])) fail(BEM_ERR_NAN, "non-finite vertex coordinate");
        ext = std::max(ext, mx[d] - mn[d]);
    }
    if (ext <= 0.0) ext = 1.0;
    t.size = ext * (1.0 + 1.0 / 1024.0);
    for (int d = 0; d < 3; ++d) t.origin[d] = 0.5 * (mn[d] + mx[d]) - 0.5 * t.size;
    for (int d = 0; d < 3; ++d) hcube[d] = t.origin[d];
    hcube[3] = 1.0 / t.size;
    if (clusters) {
        std::vector<int64_t> cvoff(c.C + 1);
        for (int64_t k = 0; k <= c.C; ++k) cvoff[k] = c.vert_off[c.cluster_boff[k]];
        DevBuf<int64_t> &dcv = t.s_i64[0];
        DevBuf<double> &cb = t.s_f64[2];
        dcv.resize(c.C + 1);
        cb.resize(6 * c.C);
        BEM_CUDA(cudaMemcpyAsync(dcv.p, cvoff.data(), (c.C + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        k_cluster_bbox<<<(unsigned)c.C, 256, 0, st>>>(dcv.p, N, c.xyz.p, cb.p);
        BEM_LAUNCH_CHECK();
        std::vector<double> hb(6 * c.C);
        BEM_CUDA(cudaMemcpyAsync(hb.data(), cb.p, hb.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        BEM_CUDA(cudaStreamSynchronize(st));
        for (int64_t k = 0; k < c.C; ++k) {
            double e = 0.0;
            for (int d = 0; d < 3; ++d) e = std::max(e, hb[6 * k + 3 + d] - hb[6 * k + d]);
            if (!(e > 0.0)) e = 1.0;
            double size = e * (1.0 + 1.0 / 1024.0);
            for (int d = 0; d < 3; ++d) hcube[4 * k + d] = 0.5 * (hb[6 * k + d] + hb[6 * k + 3 + d]) - 0.5 * size;
            hcube[4 * k + 3] = 1.0 / size;
        }
    }
    BEM_CUDA(cudaMemcpyAsync(cube.p, hcube.data(), hcube.size() * sizeof(double), cudaMemcpyHostToDevice, st));

    // 2. Morton keys at the key depth and sort
    t.key.resize(N);
    t.perm.resize(N);
    DevBuf<uint32_t> &ktmp = t.s_u32[0];
    DevBuf<int32_t> &vtmp = t.s_i32[0];
    ktmp.resize(N);
    vtmp.resize(N);
    if (clusters)
        k_keys_clusters<<<div_up(N, tb), tb, 0, st>>>(N, c.xyz.p, c.vcid.p, cube.p, t.key.p, t.perm.p);
    else
        k_keys<<<div_up(N, tb), tb, 0, st>>>(N, c.xyz.p, t.origin[0], t.origin[1], t.origin[2], 1.0 / t.size,
                                              t.key.p, t.perm.p);
    BEM_LAUNCH_CHECK();
    radix_sort_u32(t.key.p, t.perm.p, N, clusters ? 32 : 3 * kDeepLevel, ktmp.p, vtmp.p, st);

    // 3. unique boxes per level; choose l_max
    DevBuf<int32_t> &lc = t.s_i32[1];
    lc.resize(kDeepLevel + 1);
    BEM_CUDA(cudaMemsetAsync(lc.p, 0, (kDeepLevel + 1) * sizeof(int32_t), st));
    k_level_counts<<<div_up(N, tb), tb, 0, st>>>(N, t.deep, t.key.p, lc.p);
    BEM_LAUNCH_CHECK();
    int32_t hc[kDeepLevel + 1] = {};
    BEM_CUDA(cudaMemcpyAsync(hc, lc.p, (t.deep + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    BEM_CUDA(cudaStreamSynchronize(st));
    int L = 2;
    const int forced = c.level_override > 0 ? c.level_override : c.prm.fixed_level;
    if (forced > 0) {
        L = std::min(forced, t.deep);
    } else {
        for (int l = 2; l <= t.deep; ++l)
            if ((double)N / (double)(hc[l] + 1) >= (double)std::max(c.prm.leaf_target, 1)) L = l;
    }
    t.L = L;
    t.nb.assign(L + 1, 0);
    t.base.assign(L + 2, 0);
    for (int l = 0; l <= L; ++l) {
        t.nb[l] = hc[l] + 1;
        t.base[l + 1] = t.base[l] + t.nb[l];
    }
    t.nbox = t.base[L + 1];

    // 4. boxes of every level
    t.bkey.resize(t.nbox);
    t.bstart.resize(t.nbox);
    t.bcount.resize(t.nbox);
    t.parent.resize(t.nbox);
    t.leaf_of.resize(N);
    DevBuf<int32_t> &flag = t.s_i32[2], &ex = t.s_i32[3];
    flag.resize(N);
    ex.resize(N);
    int shiftL = 3 * (t.deep - L);
    k_flags_points<<<div_up(N, tb), tb, 0, st>>>(N, t.key.p, shiftL, flag.p);
    BEM_LAUNCH_CHECK();
    exclusive_scan_i32(flag.p, ex.p, N, nullptr, st);
    k_emit_leaves<<<div_up(N, tb), tb, 0, st>>>(N, t.key.p, shiftL, flag.p, ex.p, t.bkey.p + t.base[L],
                                                 t.bstart.p + t.base[L], t.leaf_of.p);
    BEM_LAUNCH_CHECK();
    for (int l = L; l >= 1; --l) {
        int n = t.nb[l];
        k_flags_boxes<<<div_up(n, tb), tb, 0, st>>>(n, t.bkey.p + t.base[l], flag.p);
        BEM_LAUNCH_CHECK();
        exclusive_scan_i32(flag.p, ex.p, n, nullptr, st);
        k_emit_parents<<<div_up(n, tb), tb, 0, st>>>(n, t.bkey.p + t.base[l], t.bstart.p + t.base[l], flag.p, ex.p,
                                                      t.bkey.p + t.base[l - 1], t.bstart.p + t.base[l - 1],
                                                      t.parent.p + t.base[l], t.base[l - 1]);
        BEM_LAUNCH_CHECK();
    }
    BEM_CUDA(cudaMemsetAsync(t.parent.p, 0xff, t.nb[0] * sizeof(int32_t), st));  // roots have no parent
    for (int l = 0; l <= L; ++l) {
        int n = t.nb[l];
        k_box_counts<<<div_up(n, tb), tb, 0, st>>>(n, t.bstart.p + t.base[l], (int32_t)N, t.bcount.p + t.base[l]);
        BEM_LAUNCH_CHECK();
    }

    // 5. near-field lists at the leaf level
    int nleaf = t.nb[L];
    t.nbr.resize((size_t)nleaf * 27);
    t.nbr_cnt.resize(nleaf);
    t.nbr_d.resize((size_t)nleaf * 27 * 4);
    DevBuf<unsigned long long> &pairs = t.s_u64[0];
    pairs.resize(1);
    BEM_CUDA(cudaMemsetAsync(pairs.p, 0, sizeof(unsigned long long), st));
    k_neighbours<<<div_up(nleaf, tb), tb, 0, st>>>(nleaf, L, t.bkey.p + t.base[L], t.bcount.p + t.base[L],
                                                    t.nbr.p, t.nbr_cnt.p, t.nbr_d.p, pairs.p);
    BEM_LAUNCH_CHECK();
    {
        DevBuf<int32_t> &ucnt = t.s_i32[4], &uoff = t.s_i32[5], &utot = t.s_i32[6];
        ucnt.resize(nleaf + 1);
        uoff.resize(nleaf + 1);
        utot.resize(1);
        k_p2p_unit_count<<<div_up(nleaf, tb), tb, 0, st>>>(nleaf, t.bcount.p + t.base[L], ucnt.p);
        BEM_LAUNCH_CHECK();
        exclusive_scan_i32(ucnt.p, uoff.p, nleaf, utot.p, st);
        int32_t nu = 0;
        BEM_CUDA(cudaMemcpyAsync(&nu, utot.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        BEM_CUDA(cudaStreamSynchronize(st));
        t.n_p2p_units = nu;
        t.p2p_units.resize(std::max<int64_t>(nu, 1));
        k_p2p_unit_emit<<<div_up(nleaf, tb), tb, 0, st>>>(nleaf, t.bcount.p + t.base[L], uoff.p, t.p2p_units.p);
        BEM_LAUNCH_CHECK();
        t.p2p_ucnt.resize(nleaf);
        BEM_CUDA(cudaMemcpyAsync(t.p2p_ucnt.p, ucnt.p, nleaf * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        // symmetric near field: per-leaf regions of the shares
        DevBuf<int32_t> &blk = t.s_i32[7], &blkoff = t.s_i32[8];
        blk.resize(nleaf + 1);
        blkoff.resize(nleaf + 1);
        t.back_S.resize(nleaf);
        t.back_base.resize(nleaf);
        t.back_gofs.resize((size_t)nleaf * 27);
        k_back_sizes<<<div_up(nleaf, tb), tb, 0, st>>>(nleaf, t.nbr.p, t.nbr_cnt.p, t.bcount.p + t.base[L], ucnt.p,
                                                        t.back_S.p, blk.p);
        BEM_LAUNCH_CHECK();
        exclusive_scan_i32(blk.p, blkoff.p, nleaf, utot.p, st);
        k_back_base<<<div_up(nleaf, tb), tb, 0, st>>>(nleaf, blkoff.p, t.back_base.p);
        BEM_LAUNCH_CHECK();
        k_back_gofs<<<div_up(nleaf, tb), tb, 0, st>>>(nleaf, t.nbr.p, t.nbr_cnt.p, t.bcount.p + t.base[L],
                                                       t.back_gofs.p);
        BEM_LAUNCH_CHECK();
        int32_t nblk = 0;
        BEM_CUDA(cudaMemcpyAsync(&nblk, utot.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        BEM_CUDA(cudaStreamSynchronize(st));
        t.n_back = 32 * (int64_t)nblk;
        t.back.resize(std::max<int64_t>(t.n_back, 1));
    }

    // 6. M2L pairs of levels 2..L, then sorted by offset class
    std::vector<int64_t> lvl_off(L + 2, 0);
    DevBuf<int32_t> &cnt = t.s_i32[9], &off = t.s_i32[10];
    std::vector<int32_t> level_tot(L + 1, 0);
    {
        size_t maxn = 0;
        for (int l = 2; l <= L; ++l) maxn = std::max<size_t>(maxn, t.nb[l]);
        cnt.resize(maxn + 1);
        off.resize(maxn + 1);
    }
    DevBuf<int32_t> &tot = t.s_i32[11];
    tot.resize(1);
    for (int l = 2; l <= L; ++l) {
        int n = t.nb[l];
        k_m2l_lists<<<div_up(n, tb), tb, 0, st>>>(n, l, t.bkey.p + t.base[l], t.bkey.p + t.base[l - 1], t.nb[l - 1],
                                                   t.base[l], 0, cnt.p, nullptr, nullptr, nullptr, nullptr);
        BEM_LAUNCH_CHECK();
        exclusive_scan_i32(cnt.p, off.p, n, tot.p, st);
        int32_t h;
        BEM_CUDA(cudaMemcpyAsync(&h, tot.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        BEM_CUDA(cudaStreamSynchronize(st));
        level_tot[l] = h;
    }
    int64_t nm2l = 0;
    for (int l = 2; l <= L; ++l) {
        lvl_off[l] = nm2l;
        nm2l += level_tot[l];
    }
    t.n_m2l = nm2l;
    DevBuf<int32_t> &ptgt = t.s_i32[12], &psrc = t.s_i32[13];
    DevBuf<uint32_t> &pcls = t.m2l_cls;  // sorted in place below: the class of every sorted pair
    ptgt.resize(nm2l);
    psrc.resize(nm2l);
    pcls.resize(std::max<int64_t>(nm2l, 1));
    for (int l = 2; l <= L; ++l) {
        int n = t.nb[l];
        if (!level_tot[l]) continue;
        k_m2l_lists<<<div_up(n, tb), tb, 0, st>>>(n, l, t.bkey.p + t.base[l], t.bkey.p + t.base[l - 1], t.nb[l - 1],
                                                   t.base[l], 0, cnt.p, nullptr, nullptr, nullptr, nullptr);
        BEM_LAUNCH_CHECK();
        exclusive_scan_i32(cnt.p, off.p, n, nullptr, st);
        k_m2l_lists<<<div_up(n, tb), tb, 0, st>>>(n, l, t.bkey.p + t.base[l], t.bkey.p + t.base[l - 1], t.nb[l - 1],
                                                   t.base[l], 1, nullptr, off.p, ptgt.p + lvl_off[l],
                                                   psrc.p + lvl_off[l], pcls.p + lvl_off[l]);
        BEM_LAUNCH_CHECK();
    }
    t.m2l_src.resize(nm2l);
    t.m2l_tgt.resize(nm2l);
    t.m2l_class_off.assign(kNumM2LClasses + 1, 0);
    if (nm2l > 0) {
        DevBuf<int32_t> &order = t.s_i32[14], &otmp = t.s_i32[15];
        DevBuf<uint32_t> &ctmp = t.s_u32[1];
        order.resize(nm2l);
        otmp.resize(nm2l);
        ctmp.resize(nm2l);
        DevBuf<int32_t> &hist = t.s_i32[16];
        hist.resize(kNumM2LClasses);
        BEM_CUDA(cudaMemsetAsync(hist.p, 0, kNumM2LClasses * sizeof(int32_t), st));
        k_hist_small<<<div_up(nm2l, tb), tb, 0, st>>>(nm2l, pcls.p, kNumM2LClasses, hist.p);
        BEM_LAUNCH_CHECK();
        k_iota<<<div_up(nm2l, tb), tb, 0, st>>>(nm2l, order.p);
        BEM_LAUNCH_CHECK();
        radix_sort_u32(pcls.p, order.p, nm2l, 9, ctmp.p, otmp.p, st);
        k_gather_i32<int32_t><<<div_up(nm2l, tb), tb, 0, st>>>(nm2l, order.p, psrc.p, t.m2l_src.p);
        k_gather_i32<int32_t><<<div_up(nm2l, tb), tb, 0, st>>>(nm2l, order.p, ptgt.p, t.m2l_tgt.p);
        BEM_LAUNCH_CHECK();
        std::vector<int32_t> hh(kNumM2LClasses);
        BEM_CUDA(cudaMemcpyAsync(hh.data(), hist.p, kNumM2LClasses * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        BEM_CUDA(cudaStreamSynchronize(st));
        for (int k = 0; k < kNumM2LClasses; ++k) t.m2l_class_off[k + 1] = t.m2l_class_off[k] + hh[k];
    }

    // 7. child -> parent pairs per level (levels 3..L), sorted by child octant
    t.up_off.assign(L + 2, 0);
    t.up_class_off.assign(L + 1, std::vector<int64_t>(9, 0));
    int64_t nup = 0;
    for (int l = 3; l <= L; ++l) {
        t.up_off[l] = nup;
        nup += t.nb[l];
    }
    t.up_off[L + 1] = nup;
    t.up_child.resize(nup);
    t.up_parent.resize(nup);
    for (int l = 3; l <= L; ++l) {
        int n = t.nb[l];
        DevBuf<uint32_t> &ok = t.s_u32[2], &oktmp = t.s_u32[3];
        DevBuf<int32_t> &id = t.s_i32[17], &idtmp = t.s_i32[18], &h8 = t.s_i32[19];
        ok.resize(n);
        oktmp.resize(n);
        id.resize(n);
        idtmp.resize(n);
        h8.resize(8);
        k_octants<<<div_up(n, tb), tb, 0, st>>>(n, t.bkey.p + t.base[l], ok.p, id.p);
        BEM_LAUNCH_CHECK();
        BEM_CUDA(cudaMemsetAsync(h8.p, 0, 8 * sizeof(int32_t), st));
        k_hist_small<<<div_up(n, tb), tb, 0, st>>>(n, ok.p, 8, h8.p);
        BEM_LAUNCH_CHECK();
        radix_sort_u32(ok.p, id.p, n, 3, oktmp.p, idtmp.p, st);
        k_up_pairs<<<div_up(n, tb), tb, 0, st>>>(n, id.p, t.base[l], t.parent.p, t.up_child.p + t.up_off[l],
                                                  t.up_parent.p + t.up_off[l]);
        BEM_LAUNCH_CHECK();
        int32_t hh[8];
        BEM_CUDA(cudaMemcpyAsync(hh, h8.p, sizeof(hh), cudaMemcpyDeviceToHost, st));
        BEM_CUDA(cudaStreamSynchronize(st));
        for (int k = 0; k < 8; ++k) t.up_class_off[l][k + 1] = t.up_class_off[l][k] + hh[k];
    }

    // 8. target-major CSR of the M2L and child->parent pairs (stable: ascending pair index)
    auto target_csr = [&](const int32_t *tgt, int64_t np, DevBuf<int32_t> &off, DevBuf<int32_t> &by) {
        off.resize((size_t)t.nbox + 1);
        by.resize(np > 0 ? np : 1);
        DevBuf<int32_t> &cnt2 = t.s_i32[20];
        cnt2.resize((size_t)t.nbox + 1);
        BEM_CUDA(cudaMemsetAsync(cnt2.p, 0, ((size_t)t.nbox + 1) * sizeof(int32_t), st));
        if (np > 0) {
            DevBuf<uint32_t> &k = t.s_u32[4], &ktmp2 = t.s_u32[5];
            DevBuf<int32_t> &vtmp2 = t.s_i32[21];
            k.resize(np);
            ktmp2.resize(np);
            vtmp2.resize(np);
            k_copy_keys<<<div_up(np, tb), tb, 0, st>>>(np, tgt, k.p, cnt2.p);
            BEM_LAUNCH_CHECK();
            k_iota<<<div_up(np, tb), tb, 0, st>>>(np, by.p);
            BEM_LAUNCH_CHECK();
            int bits = 1;
            while ((1ll << bits) <= (long long)t.nbox) ++bits;
            radix_sort_u32(k.p, by.p, np, bits, ktmp2.p, vtmp2.p, st);
        }
        exclusive_scan_i32(cnt2.p, off.p, (int64_t)t.nbox + 1, nullptr, st);
    };
    target_csr(t.m2l_tgt.p, nm2l, t.m2l_tgt_off, t.m2l_by_tgt);
    target_csr(t.up_parent.p, nup, t.up_par_off, t.up_by_par);

    // 9. sorted point data
    t.loc64.resize(3 * N);
    t.loc32.resize(3 * N);
    t.nrm64.resize(3 * N);
    t.nrm32.resize(3 * N);
    t.s_sorted.resize(N);
    t.ih.resize(N);
    k_sorted_points<<<div_up(N, tb), tb, 0, st>>>(N, L, t.deep, t.perm.p, t.key.p, c.xyz.p, c.nrm.p, c.s.p, cube.p,
                                                   clusters ? c.vcid.p : nullptr, t.loc64.p, t.loc32.p, t.nrm64.p,
                                                   t.nrm32.p, t.s_sorted.p, t.ih.p);
    BEM_LAUNCH_CHECK();
    unsigned long long hpairs = 0;
    BEM_CUDA(cudaMemcpyAsync(&hpairs, pairs.p, sizeof(hpairs), cudaMemcpyDeviceToHost, st));
    BEM_CUDA(cudaStreamSynchronize(st));
    t.p2p_pairs = (int64_t)hpairs;
}

}  // namespace bem
