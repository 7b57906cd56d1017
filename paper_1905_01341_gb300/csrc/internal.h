// Internal declarations shared by the CUDA translation units of libbem.so.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "bem.h"

namespace bem {

// ------------------------------------------------------------------------------ errors
struct Error {
    int code;
    std::string msg;
};

[[noreturn]] inline void fail(int code, const std::string &msg) { throw Error{code, msg}; }

#define BEM_CUDA(expr)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess)                                                             \
            ::bem::fail(e_ == cudaErrorMemoryAllocation ? BEM_ERR_NOMEM : BEM_ERR_CUDA,    \
                        std::string(#expr) + " -> " + cudaGetErrorString(e_) + " at " +    \
                            __FILE__ + ":" + std::to_string(__LINE__));                    \
    } while (0)

// Message of the last failure that has no context (bem_create, context-free entry points),
// returned by bem_last_error(NULL); one per host thread.
extern thread_local std::string g_create_error;

// Every kernel launch of the library is followed by this check, which also counts it.
extern long long g_launch_count;
#define BEM_LAUNCH_CHECK()                 \
    do {                                   \
        ++::bem::g_launch_count;           \
        BEM_CUDA(cudaGetLastError());      \
    } while (0)

// ------------------------------------------------------------------------------ device buffers
// Grow-only device allocation; never shrinks, so repeated builds of the same size reuse it.
template <class T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0, cap = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    void resize(size_t m) {
        if (m > cap) {
            if (p) cudaFree(p);
            p = nullptr;
            cap = 0;
            size_t bytes = (m ? m : 1) * sizeof(T);
            BEM_CUDA(cudaMalloc(&p, bytes));
            cap = m;
        }
        n = m;
    }
    T *get() const { return p; }
};

// Pinned host scratch for small device->host reads.
template <class T>
struct HostPinned {
    T *p = nullptr;
    size_t cap = 0;
    HostPinned(const HostPinned &) = delete;
    HostPinned &operator=(const HostPinned &) = delete;
    HostPinned() = default;
    ~HostPinned() {
        if (p) cudaFreeHost(p);
    }
    T *get(size_t m) {
        if (m > cap) {
            if (p) cudaFreeHost(p);
            p = nullptr;
            BEM_CUDA(cudaMallocHost(&p, (m ? m : 1) * sizeof(T)));
            cap = m;
        }
        return p;
    }
};

inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }

constexpr int kMaxRhs = 4;
constexpr int kDeepLevel = 10;       // Morton keys are computed at this depth (30 bits)
constexpr int kMaxPfmm = 20;
// largest bubble (vertices; icosphere level 4) for which the automatic mode runs the diagonal
// product's M2L on the tensor cores
constexpr int64_t kDiagTcMaxVerts = 2562;
constexpr int kNumM2LClasses = 316;  // offsets in [-3,3]^3 minus the 27 near ones

// ------------------------------------------------------------------------------ octree
struct Tree {
    int L = 0;                 // leaf level l_max
    int deep = kDeepLevel;     // depth of the point keys (8 when the key carries a cluster id)
    DevBuf<double> ih;         // [N] 1 / (leaf box size) of each sorted point's cluster
    double origin[3] = {0, 0, 0};
    double size = 1.0;         // bounding cube edge
    int64_t N = 0;
    DevBuf<int32_t> perm;      // sorted position -> caller vertex index
    DevBuf<uint32_t> key;      // deep Morton keys of sorted points
    // boxes of all levels 0..L, concatenated level by level
    std::vector<int> nb;       // boxes per level
    std::vector<int> base;     // first global box index of each level
    int nbox = 0;
    DevBuf<uint32_t> bkey;     // Morton key of a box at its own level
    DevBuf<int32_t> bstart;    // first sorted point of the box
    DevBuf<int32_t> bcount;    // points in the box
    DevBuf<int32_t> parent;    // global index of the parent box (-1 at level 0)
    DevBuf<int32_t> leaf_of;   // leaf box (level-local index) of every sorted point
    // near field: for every leaf, up to 27 neighbour leaves (self included)
    DevBuf<int32_t> nbr;       // [nleaf][27] level-local leaf indices
    DevBuf<int32_t> nbr_cnt;   // [nleaf]
    DevBuf<int8_t> nbr_d;      // [nleaf][27][4] offset (dx,dy,dz) in leaf boxes
    // M2L: pairs of all levels sorted by offset class
    int64_t n_m2l = 0;
    DevBuf<int32_t> m2l_src, m2l_tgt;  // global box indices
    DevBuf<uint32_t> m2l_cls;          // offset class of each pair (ascending)
    std::vector<int64_t> m2l_class_off;  // [kNumM2LClasses+1] host copy
    // M2M / L2L: per level l (1..L), child->parent pairs sorted by child octant
    std::vector<int64_t> up_off;       // per level: offset into up_child/up_parent
    std::vector<std::vector<int64_t>> up_class_off;  // per level: [9]
    DevBuf<int32_t> up_child, up_parent;
    // target-major views of the pair lists, for the fixed-order reductions: for every box,
    // the pair indices that write to it, ascending (CSR over all boxes)
    DevBuf<int32_t> m2l_tgt_off, m2l_by_tgt;  // [nbox+1], [n_m2l]
    DevBuf<int32_t> up_par_off, up_by_par;    // [nbox+1], [n_up]
    // leaf-local coordinates of sorted points in units of the leaf box (range [-1/2, 1/2))
    DevBuf<double> loc64;      // [3][N]
    DevBuf<float> loc32;       // [3][N]
    DevBuf<double> nrm64;      // [3][N] sorted normals
    DevBuf<float> nrm32;
    DevBuf<double> s_sorted;   // [N]
    int64_t p2p_pairs = 0;
    // near-field work units: (leaf, first receiver), up to 64 receivers of one leaf each
    DevBuf<int2> p2p_units;
    int64_t n_p2p_units = 0;
    DevBuf<int32_t> p2p_ucnt;  // [nleaf] units per leaf
    // symmetric near field (FP32 single-RHS products): a pair of neighbour leaves A < B is
    // evaluated once, by A's units; each unit of A writes B's share (one float per point of B)
    // into its own region of `back`, and a gather adds those shares to B's points in a fixed order
    DevBuf<int32_t> back_S;     // [nleaf] floats one unit of leaf A writes (its neighbours B > A)
    DevBuf<int64_t> back_base;  // [nleaf] first float of leaf A's units' region
    DevBuf<int32_t> back_gofs;  // [nleaf][27] neighbour k = A < B of leaf B: offset of B's share in a unit of A; else -1
    DevBuf<float> back;         // [n_back]
    int64_t n_back = 0;
    // scratch of the build, kept between builds so that a rebuild allocates (and synchronises)
    // nothing once the sizes have settled; each slot has one use
    DevBuf<int32_t> s_i32[22];
    DevBuf<uint32_t> s_u32[6];
    DevBuf<int64_t> s_i64[1];
    DevBuf<double> s_f64[3];
    DevBuf<unsigned long long> s_u64[1];
};

// ------------------------------------------------------------------------------ FMM operators
struct Operators {
    bool ready = false;
    int p = 0, P = 0;
    DevBuf<double> m2l64, m2m64, l2l64;  // [316][P][P], [8][P][P], [8][P][P]
    DevBuf<float> m2l32, m2m32, l2l32;
    // tensor-core M2L: per class, per 16-wide K step, three BF16 pieces of an N_pad x 16 block
    // in the K-major core-matrix layout (m2l_tc.cu); stored as raw 16-bit words
    int tc_Npad = 0, tc_Kpad = 0;
    DevBuf<uint16_t> m2l_tc;
    // per-class M2L truncation: class c translates the coefficients of degrees < p_c, padded to
    // the 16-wide steps of the products: cls_K[c] = 16 * ceil(p_c^2 / 16), capped at the full
    // padded size (margin < 0: every class at p)
    int margin = -1;
    std::vector<int> cls_p, cls_Kh;  // per class: order p_c, truncated size K_c (host copies)
    DevBuf<int32_t> cls_K;
};

// Work chunk of the class-grouped translation product.
struct XChunk {
    int32_t cls;     // matrix index
    int32_t count;   // pairs in the chunk
    int64_t start;   // first pair
};

// ------------------------------------------------------------------------------ profiling
// Phases timed with CUDA events on the context's stream when profiling is enabled.
enum Phase {
    PH_GEOMETRY = 0,
    PH_TREE,
    PH_OPERATORS,
    PH_STRENGTHS,
    PH_P2M,
    PH_M2M,
    PH_M2L,
    PH_L2L,
    PH_L2P,
    PH_P2P,
    PH_DIRECT,
    PH_DIAG,
    PH_GMRES,
    PH_M2L_REDUCE,  // per-target sums of the M2L pair products
    PH_M2L_CC,      // M2L translations on the CUDA cores (FP64 path, 4-RHS diagonal product)
    PH_COUNT
};

struct Profiler {
    bool on = false;
    struct Rec {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<cudaEvent_t> pool;
    std::vector<Rec> recs;
    cudaEvent_t take() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        BEM_CUDA(cudaEventCreate(&e));
        return e;
    }
    ~Profiler() {
        for (auto &r : recs) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

// Per-shape least-squares spherical-harmonic basis (Eqs. (3.22)-(3.23)): for every distinct
// initial bubble shape, G [nd][Pf] and G+ = (G^T G)^(-1) G^T [Pf][nd], concatenated.
// Bubbles whose vertex directions from their centroid coincide (same vertex count and
// order) share one shape; `rep` is the first bubble of the shape.
struct BubbleShape {
    int64_t rep;
    int nd;
    double cx, cy, cz;  // centroid of the representative
};

struct ShBasis {
    int pf = 0, Pf = 0;
    DevBuf<double> G, Gp;
    DevBuf<float2> Gs, Gps;    // G transposed ([Pf][nd] per shape) and G+ as FP32 (hi, lo) pairs
    DevBuf<int64_t> g_off;     // per shape offset (elements) into G / Gp
    DevBuf<int32_t> shape_of;  // [M] shape index of each bubble
};

struct Context;
struct StepState;
struct Mlp;
void step_free(StepState *s);
void mlp_free(Mlp *m);
// Records the device time of everything launched on the context stream during its lifetime.
struct PhaseScope {
    Context *c;
    int phase;
    cudaStream_t s;  // the stream the phase's kernels run on
    cudaEvent_t a = nullptr;
    PhaseScope(Context &cc, int ph);
    PhaseScope(Context &cc, int ph, cudaStream_t st);
    ~PhaseScope();
};

// ------------------------------------------------------------------------------ context
struct Context {
    bem_params prm{};
    cudaStream_t stream = nullptr;
    // streams of the FMM product: after the strengths, the near field and the far field run
    // concurrently on two internal streams and join back into `stream` (created on first use)
    cudaStream_t side = nullptr, hi = nullptr;  // near field (lowest priority), far field (highest)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_far = nullptr, ev_m2l = nullptr;
    int device = 0;
    std::string err;

    int64_t N = 0, T = 0, M = 0;
    DevBuf<double> xyz;      // [3][N]
    DevBuf<int32_t> tri;     // [3][T]
    std::vector<int64_t> vert_off, tri_off;
    DevBuf<int32_t> v2t_off, v2t;  // vertex -> triangle CSR (sorted triangle ids)
    bool mesh_ok = false;
    bool points_only = false;      // bem_points_upload: unit weights, no triangles, no diagonals
    // independent clusters (bem_mesh_set_clusters): cluster c owns bubbles
    // cluster_boff[c]..cluster_boff[c+1]-1; no interaction crosses clusters
    int64_t C = 1;
    std::vector<int64_t> cluster_boff;
    // octree depth: level_override > 0 forces l_max (depth autotuning); tuned_level is the
    // depth the autotuner chose for this mesh (0 = not tuned yet)
    int level_override = 0, tuned_level = 0;
    // tile choices of the products: tensor-core M2L pipeline stages (0 = deepest that fits) and
    // near-field blocks per SM (0 = one warp per unit); set from the parameters, or by the
    // autotuner when those are automatic
    int tuned_stages = 0, tuned_p2p_blocks = 0, tuned_overlap = 1;
    int num_sms = 1;
    DevBuf<int32_t> vcid;          // [N] cluster of every vertex (when C > 1)

    // geometry (caller order)
    DevBuf<double> s, nrm;         // [N], [3][N]
    DevBuf<double> ldiag, mdiag;   // [N]
    bool built = false;

    Tree tree;
    Operators ops;
    Operators ops_diag;  // operators of the 4-RHS diagonal product when diag_p_fmm != p_fmm

    // FMM work arrays
    DevBuf<double> q64, w64;       // strengths [R][N] sorted order
    DevBuf<float> q32, w32;
    DevBuf<double> mp64, lc64;     // expansions [nbox][R][P]
    DevBuf<float> mp32, lc32;
    DevBuf<int32_t> m2l_byK;       // truncated row length of each M2L pair, target-major order
    DevBuf<double> ypair64;        // per-pair translation results [pair][R][P]
    DevBuf<float> ypair32;
    DevBuf<double> far64;          // far-field potential [R][N] (sorted)
    DevBuf<float> far32;
    DevBuf<double> near_out;       // combined potential [R][N] (sorted)
    DevBuf<XChunk> m2l_chunks;
    std::vector<XChunk> m2l_chunks_h;
    // M2L chunks of <= 256/R pairs for the tensor-core kernel: [0] for R = 1, [1] for R = 4
    DevBuf<XChunk> tc_chunks[2];
    bool tc_chunks_ok[2] = {false, false};  // built for the current tree
    bool diag_tc = false;                     // the 4-RHS diagonal product uses the tensor-core M2L
    int64_t n_tc_chunks[2] = {0, 0};
    DevBuf<uint16_t> xsplit;         // multipoles split into three BF16 planes (tensor-core M2L)
    // target-major tensor-core M2L, one state per RHS count R (index 0: R = 1, index 1: R = 4;
    // the products use R = 1, the 4-RHS diagonal product the pair-major kernel): target boxes
    // grouped by octant into tiles of 256 / R targets (256 rows of (target, rhs)); per tile the
    // offset classes present, by truncated size (ascending), cut into items of a few classes;
    // each item's partial local expansions, summed per target
    struct TmState {
        bool ok = false;                 // built for the current tree and the operators `ops`
        const Operators *ops = nullptr;
        int64_t ntiles = 0, nitems = 0;
        DevBuf<int32_t> box;             // [tiles * 256 / R] global box index of each tile slot, -1 past the end
        DevBuf<int32_t> src;             // [tiles][316][256 / R] source box of each (tile, class, slot), -1 if none
        DevBuf<int32_t> cls;             // [tiles][316] the tile's classes, truncated size ascending
        DevBuf<int32_t> item_off;        // [tiles + 1] first item of each tile
        DevBuf<int4> items;              // [items] (tile, first class slot, classes, largest truncated size)
        DevBuf<float> part;              // [items][256][N_pad] partial local expansions
        DevBuf<int32_t> s_i32[8];        // scratch of the table build (kept between builds)
        DevBuf<uint32_t> s_u32[2];
    };
    TmState tm[2];
    DevBuf<int> tc_err;              // set by a tensor-core block whose wait ran out
    DevBuf<double2> tri_tmp;         // [2T] per-triangle pairs: area vectors, then (n x v)_k A_k
    // per-build and per-step scratch kept in the context (a cudaFree synchronises the device):
    // flags of the finiteness and mesh checks, one per check site, and the diagonal product's output
    DevBuf<int> chk[4];
    DevBuf<double> diag_tmp;
    std::vector<DevBuf<XChunk> *> up_chunks;  // per level
    std::vector<std::vector<XChunk>> up_chunks_h;
    DevBuf<double> ones;

    // direct-sum work arrays
    DevBuf<float> dir_hi, dir_lo;  // [3][N] split coordinates
    double dir_centre[3] = {0, 0, 0};

    // staging for host pointers
    DevBuf<double> stage_in[4];
    DevBuf<double> stage_out;

    // GMRES
    DevBuf<double> V, wv, rv, bv, zv, hcol, hmat, givens, gvec, yvec, partial, scal;
    DevBuf<double> dv;   // a GMRES cycle's update d = P V y
    DevBuf<float> V32;   // the Krylov basis in FP32 (mixed precision)
    DevBuf<double> vk64; // the current basis vector of V32 in FP64, the product's input
    // bubble-block preconditioner (gmres_precond = 2, precond.cu): per distinct bubble mesh
    // (connectivity), the inverse of the isolated representative's single-layer block at unit
    // size, built from the geometry of the first solve after a mesh upload
    struct BlockPrecond {
        bool ready = false;
        std::vector<int> nd;              // vertices per shape
        std::vector<int64_t> inv_off;     // [shapes + 1] offsets (elements) into inv64
        std::vector<int64_t> first;       // [shapes + 1] offsets into the grouped bubble lists
        DevBuf<double> inv64;             // row-major nd x nd per shape, unit size
        std::vector<int64_t> tc_off;      // [shapes + 1] offsets (elements) into tcA
        DevBuf<uint16_t> tcA;             // per shape the inverse as three BF16 pieces, K-major blocks
        bool tc_attr = false;             // the tensor-core apply's shared-memory size is set
        DevBuf<int64_t> bub_voff;         // [M] first vertex of each bubble, grouped by shape
        DevBuf<double> bub_scale;         // [M] 1 / (mean centroid distance) at the current geometry
        DevBuf<uint16_t> ys;              // the right-hand side as three BF16 pieces (mixed precision)
    } bp;
    HostPinned<double> hscal;
    // GMRES of independent clusters (gmres_batched.cu): reduction segments and per-cluster state
    struct BatchedGmres {
        int C = 0, nseg = 0;
        int64_t N = 0;
        DevBuf<int64_t> s0, s1;
        DevBuf<int32_t> seg_off, active, sel, kk;
        DevBuf<double> partial, h, h2, H, cs, sn, g, y, nrm2, res;
    } gb;
    // per cluster, for the last solve: GMRES iterations, true relative residual, device ms from
    // the start of the solve until the cluster's solution was final; and the solve's device ms
    std::vector<int> cl_iters;
    std::vector<double> cl_relres, cl_done_ms;
    double cl_solve_ms = 0.0;
    std::vector<cudaEvent_t> cl_events;
    int cl_events_used = 0;

    bem_stats stats{};
    std::vector<double> res_hist;  // residual estimates |g_{k+1}|/|b| of the last solve
    StepState *step = nullptr;     // time-integration state (timestep.cu)
    Mlp *mlp = nullptr;            // learned initial guess (mlp.cu)
    DevBuf<int64_t> voff_d;        // [M+1] device copy of vert_off
    Profiler prof;
    ~Context();
};

// ------------------------------------------------------------------------------ cross-TU entry points
// geometry.cu
void build_vertex_triangle_csr(Context &c);
void compute_vertex_geometry(Context &c);

// tree.cu
void build_tree(Context &c);
void radix_sort_u32(uint32_t *keys, int32_t *vals, int64_t n, int bits, uint32_t *keys_tmp,
                    int32_t *vals_tmp, cudaStream_t st);
void exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *total_dev,
                        cudaStream_t st);

// fmm.cu
void build_operators(Context &c, Operators &o, int p);
// truncation order of each M2L offset class for expansion order p (bem_params.m2l_order_margin)
std::vector<int> m2l_class_orders(int p, int margin);
// out[r][i] (caller order) = sum over the R right-hand sides of the off-diagonal product:
// f[r] (L_off xL[r]) + g[r] (M_off xM[r]); prec = bem_precision.
void offdiag_apply(Context &c, int R, const double *f, const double *const *xL,
                   const double *g, const double *const *xM, double *const *out, int prec,
                   const Operators *ops = nullptr);

// p2p.cu
template <class T, int R>
void launch_p2p_list(Context &c, const T *q, const T *w, double *near_sorted, bool hq, bool hw, cudaStream_t st);
template <int R>
void launch_direct(Context &c, int prec, const double *f, const double *const *xL,
                   const double *g, const double *const *xM, double *const *out);

// Direct FP32 product (k_direct32, one right-hand side) on caller-provided split coordinates.
void launch_direct32_raw(int64_t N, const float *hi, const float *lo, const double *s, const double *nrm, double f,
                         const double *xL, double g, const double *xM, double *out, cudaStream_t st);

// m2l_tc.cu
bool m2l_tc_supported(int P);
void build_tc_tables(Context &c, Operators &o);
template <int R>
void launch_m2l_tc(Context &c, const Operators &o, const XChunk *chunks, int64_t nchunks, const float *X, int64_t xrows, float *Ypair,
                   int *err, cudaStream_t st);
int m2l_tc_pairs_per_chunk(int R, int Kc);
// target-major form (R = 1 or 4 right-hand sides): the items' partial local expansions, then
// (reduce) the locals lc[box][R][P] of every M2L target = its partials summed
template <int R>
void launch_m2l_tm(Context &c, const Operators &o, const float *X, int64_t xrows, int *err, cudaStream_t st);
template <int R>
void launch_m2l_tm_reduce(Context &c, const Operators &o, float *lc, cudaStream_t st);

// gmres.cu, gmres_batched.cu (clusters: one GMRES per cluster, in lockstep)
void gmres_solve(Context &c, const double *b, double *x, int *iters, double *relres);
void gmres_solve_batched(Context &c, const double *b, double *x, int *iters, double *relres);

inline PhaseScope::PhaseScope(Context &cc, int ph) : PhaseScope(cc, ph, cc.stream) {}
inline PhaseScope::PhaseScope(Context &cc, int ph, cudaStream_t st) : c(&cc), phase(ph), s(st) {
    if (c->prof.on) {
        a = c->prof.take();
        BEM_CUDA(cudaEventRecord(a, s));
    }
}
inline PhaseScope::~PhaseScope() {
    if (a) {
        cudaEvent_t b = c->prof.take();
        cudaEventRecord(b, s);
        c->prof.recs.push_back({phase, a, b});
    }
}

// bem_api.cu
// out[i] += f ld[i] xL[i] + g md[i] xM[i] (the identity diagonals of Eqs. (s3), (s5))
void launch_add_diag(int64_t N, double f, const double *xL, double g, const double *xM, const double *ld,
                     const double *md, double *out, cudaStream_t st);
// hi[i] = fp32(x[i]), lo[i] = fp32(x[i] - hi[i]) (coordinates of the FP32 direct product)
void launch_split_hilo(int64_t n, const double *x, float *hi, float *lo, cudaStream_t st);
void apply_full(Context &c, double f, const double *xL, double g, const double *xM, double *out);
void build_all(Context &c);
void solve_internal(Context &c, const double *phi, double *q, int *it, double *rr);
bool is_device_ptr(const Context &c, const void *p);

// timestep.cu
void step_init(Context &c, const double *phi0_dev, const double *q0_dev, const bem_step_params &sp);
void step_advance(Context &c, bem_step_stats &st);
void step_get_state(Context &c, double *xyz, double *phi, double *q, double *t);
void step_set_state(Context &c, const double *xyz, const double *phi, const double *q);
void step_filter(Context &c, const double *x, double *y);
int64_t step_checkpoint_size(const Context &c);
void step_save(Context &c, void *buf, int64_t cap);
void step_load(Context &c, const void *buf, int64_t size);
void build_sh_basis(Context &c, int pf, ShBasis &B, int *bad, const double *xyz = nullptr, bool allow_torus = false);
// Groups the bubbles by shape from host coordinates hx [3][N] (timestep.cu).
void find_shapes(const Context &c, const std::vector<double> &hx, std::vector<BubbleShape> &shapes,
                 std::vector<int32_t> &shape_of);
// precond.cu: bubble-block preconditioner of GMRES
void block_precond_prepare(Context &c);                     // build once, refresh the per-bubble scales
void block_precond_apply(Context &c, const double *y, double *z);  // z = P y
void block_precond_check(Context &c);  // fails with BEM_ERR_TIMEOUT if a tensor-core wait ran out
const double *step_initial_xyz(Context &c);

// mlp.cu
struct MlpStats {
    int64_t solves = 0;          // solves that used the learned guess
    int64_t iters_guess = 0;     // their GMRES iterations
    int64_t iters_fallback = 0;  // iterations of the same solves from q_prev (compare mode)
    double res0_guess = 0.0;     // summed initial relative residuals of each start
    double res0_fallback = 0.0;
};
void mlp_init(Context &c, int hidden, int lmax, uint64_t seed, const double *xyz0);
void mlp_set_mode(Context &c, int record, int use, int compare);
bool mlp_active(Context &c);
bool mlp_compare(Context &c);
void mlp_before_solve(Context &c, const double *phi, double *q, bool uniform);
const double *mlp_qprev(Context &c);
void mlp_after_solve(Context &c, const double *q);
double mlp_train(Context &c, int epochs, int batch, double lr);
double mlp_loss_grad(Context &c, int B, const double *F, const double *T, double *grads_dev);
void mlp_forward(Context &c, int B, const double *F, double *Y);
void mlp_get_params(Context &c, double *out);
void mlp_set_params(Context &c, const double *in);
int64_t mlp_samples(Context &c);
int64_t mlp_num_params(const Mlp &m);
const int *mlp_dims(Context &c);
MlpStats &mlp_stats(Context &c);

}  // namespace bem
