// C ABI of libbem.so (declared in include/bem.h): context management, mesh upload, build,
// operator products, right-hand side and the GMRES solve. Host or device pointers are
// accepted for every array; host arrays are staged through context-owned device buffers.
#include "internal.h"

#include <cmath>
#include <cstring>
#include <exception>

namespace bem {

long long g_launch_count = 0;

Context::~Context() {
    for (auto e : cl_events) cudaEventDestroy(e);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (ev_far) cudaEventDestroy(ev_far);
    if (ev_m2l) cudaEventDestroy(ev_m2l);
    if (side) cudaStreamDestroy(side);
    if (hi) cudaStreamDestroy(hi);
    for (auto *p : up_chunks) delete p;
    step_free(step);
    mlp_free(mlp);
}

bool is_device_ptr(const Context &c, const void *p) {
    if (!p) return false;
    cudaPointerAttributes a{};
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
        if (a.type == cudaMemoryTypeDevice && a.device != c.device)
            fail(BEM_ERR_ARG, "device pointer belongs to another device");
        return true;
    }
    return false;
}

thread_local std::string g_create_error;

namespace {

__global__ void k_add_diag(int64_t N, double f, const double *__restrict__ xL, double g,
                           const double *__restrict__ xM, const double *__restrict__ ld,
                           const double *__restrict__ md, double *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double v = out[i];
    if (f != 0.0) v += f * ld[i] * xL[i];
    if (g != 0.0) v += g * md[i] * xM[i];
    out[i] = v;
}

// Eq. (s3): M_ii = -1/2 - (M_off 1)_i.  Eq. (s5): L_ii = n_i . [v_i + (1/2 + M_ii) r_i] with
// v_i = sum_{j != i} (M_ij r_j - L_ij n_j) componentwise.
__global__ void k_diag_identities(int64_t N, const double *__restrict__ d0, const double *__restrict__ vx,
                                  const double *__restrict__ vy, const double *__restrict__ vz,
                                  const double *__restrict__ xyz, const double *__restrict__ nrm,
                                  double *__restrict__ ld, double *__restrict__ md) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double m = -0.5 - d0[i];
    double a = 0.5 + m;
    md[i] = m;
    ld[i] = nrm[i] * (vx[i] + a * xyz[i]) + nrm[N + i] * (vy[i] + a * xyz[N + i]) +
            nrm[2 * N + i] * (vz[i] + a * xyz[2 * N + i]);
}

__global__ void k_fill(int64_t N, double v, double *a) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N) a[i] = v;
}

__global__ void k_split(int64_t N, const double *__restrict__ x, float *__restrict__ hi, float *__restrict__ lo) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    float h = (float)x[i];
    hi[i] = h;
    lo[i] = (float)(x[i] - (double)h);
}

__global__ void k_rhs_combine(int64_t N, const double *__restrict__ phi, double *__restrict__ b) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N) b[i] += -0.5 * phi[i];
}

__global__ void k_check_finite(int64_t N, const double *__restrict__ a, int *__restrict__ bad) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N && !isfinite(a[i])) atomicOr(bad, 1);
}

Context *as_ctx(void *p) {
    if (!p) fail(BEM_ERR_ARG, "null context");
    return static_cast<Context *>(p);
}

// Device view of an input vector of length n (copies host arrays into stage buffer k).
const double *dev_in(Context &c, const double *p, int64_t n, int k) {
    if (!p) return nullptr;
    if (is_device_ptr(c, p)) return p;
    c.stage_in[k].resize(n);
    BEM_CUDA(cudaMemcpyAsync(c.stage_in[k].p, p, n * sizeof(double), cudaMemcpyHostToDevice, c.stream));
    return c.stage_in[k].p;
}

struct OutView {
    Context &c;
    double *user;
    double *dev;
    int64_t n;
    bool host;
    OutView(Context &cc, double *p, int64_t nn) : c(cc), user(p), n(nn) {
        if (!p) fail(BEM_ERR_ARG, "null output");
        host = !is_device_ptr(c, p);
        if (host) {
            c.stage_out.resize(n);
            dev = c.stage_out.p;
        } else {
            dev = p;
        }
    }
    void finish() {
        if (host) {
            BEM_CUDA(cudaMemcpyAsync(user, dev, n * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
            BEM_CUDA(cudaStreamSynchronize(c.stream));
        }
    }
};

void require_built(Context &c) {
    if (!c.mesh_ok) fail(BEM_ERR_NOT_BUILT, "no mesh uploaded");
    if (!c.built) fail(BEM_ERR_NOT_BUILT, "fmm_build has not been called since the last mesh change");
}

template <class F>
int guarded(void *ctx, F &&fn) {
    Context *c = nullptr;
    try {
        c = as_ctx(ctx);
        c->err.clear();
        BEM_CUDA(cudaSetDevice(c->device));
        fn(*c);
        return BEM_OK;
    } catch (const Error &e) {
        if (c) c->err = e.msg;
        else g_create_error = e.msg;
        return e.code;
    } catch (const std::exception &e) {
        if (c) c->err = e.what();
        return BEM_ERR_CUDA;
    }
}

void check_params(const bem_params &p) {
    if (p.p_fmm < 2 || p.p_fmm > kMaxPfmm) fail(BEM_ERR_ARG, "p_fmm must be in 2..20");
    if (p.leaf_target < 0) fail(BEM_ERR_ARG, "leaf_target must be >= 0 (0 = autotune the depth)");
    if (p.fixed_level < 0 || p.fixed_level > kDeepLevel || p.fixed_level == 1)
        fail(BEM_ERR_ARG, "fixed_level must be 0 or in 2..10");
    if (p.precision != BEM_PREC_FP64 && p.precision != BEM_PREC_MIXED) fail(BEM_ERR_ARG, "bad precision");
    if (p.diag_precision != -1 && p.diag_precision != BEM_PREC_FP64 && p.diag_precision != BEM_PREC_MIXED)
        fail(BEM_ERR_ARG, "bad diag_precision");
    if (p.diag_p_fmm != -1 && (p.diag_p_fmm < 2 || p.diag_p_fmm > kMaxPfmm))
        fail(BEM_ERR_ARG, "diag_p_fmm must be -1 or in 2..20");
    if (p.overlap < -1 || p.overlap > 2) fail(BEM_ERR_ARG, "overlap must be -1, 0, 1 or 2");
    if (p.mvp != BEM_MVP_FMM && p.mvp != BEM_MVP_DIRECT) fail(BEM_ERR_ARG, "bad mvp kind");
    if (p.m2l_tensor_cores < 0 || p.m2l_tensor_cores > 3) fail(BEM_ERR_ARG, "m2l_tensor_cores must be 0..3");
    if (p.gmres_maxit < 1 || p.gmres_restart < 0 || p.gmres_restart > 127) fail(BEM_ERR_ARG, "bad GMRES limits");
    if (p.gmres_precond < 0 || p.gmres_precond > 2) fail(BEM_ERR_ARG, "gmres_precond must be 0, 1 or 2");
    if (!(p.gmres_tol > 0.0)) fail(BEM_ERR_ARG, "gmres_tol must be > 0");
    if (p.m2l_stages != 0 && (p.m2l_stages < 2 || p.m2l_stages > 3)) fail(BEM_ERR_ARG, "m2l_stages must be 0, 2 or 3");
    if (p.p2p_blocks_per_sm < -1 || p.p2p_blocks_per_sm > 16) fail(BEM_ERR_ARG, "p2p_blocks_per_sm must be in -1..16");
    if (p.m2l_order_margin < -1 || p.m2l_order_margin > 20) fail(BEM_ERR_ARG, "m2l_order_margin must be in -1..20");
    if (p.m2l_target_major != 0 && p.m2l_target_major != 1) fail(BEM_ERR_ARG, "m2l_target_major must be 0 or 1");
}

}  // namespace

void launch_add_diag(int64_t N, double f, const double *xL, double g, const double *xM, const double *ld,
                     const double *md, double *out, cudaStream_t st) {
    k_add_diag<<<div_up(N, 256), 256, 0, st>>>(N, f, xL, g, xM, ld, md, out);
    BEM_LAUNCH_CHECK();
}

void launch_split_hilo(int64_t n, const double *x, float *hi, float *lo, cudaStream_t st) {
    k_split<<<div_up(n, 256), 256, 0, st>>>(n, x, hi, lo);
    BEM_LAUNCH_CHECK();
}

// out = f (L_off + diag(Ldiag)) xL + g (M_off + diag(Mdiag)) xM, all device pointers.
void apply_full(Context &c, double f, const double *xL, double g, const double *xM, double *out) {
    double fa[1] = {f}, ga[1] = {g};
    const double *xl[1] = {xL};
    const double *xm[1] = {xM};
    double *o[1] = {out};
    offdiag_apply(c, 1, fa, xl, ga, xm, o, c.prm.precision);
    launch_add_diag(c.N, f, xL, g, xM, c.ldiag.p, c.mdiag.p, out, c.stream);
}

// Tile autotuner (leaf_target = 0). Times one single-layer product at the depth the leaf-count
// rule gives for 64 points per leaf and at one level either side, and keeps the fastest depth
// for this mesh: points on surfaces fill ~4x more boxes per level, not 8x, so the near-field /
// far-field balance moves in coarse steps and is cheapest to settle by timing. At that depth it
// then times the tile choices left automatic: the tensor-core M2L's pipeline depth (3, 4 or 5
// shared-memory stages) and the near field's grid (one warp per unit, or a persistent grid of
// k blocks per SM). Both decide how the near field and the far field share the SMs while they
// run concurrently on two streams; neither changes a result.
void tune_tiles(Context &c) {
    const int64_t N = c.N;
    c.ones.resize(N);
    k_fill<<<div_up(N, 256), 256, 0, c.stream>>>(N, 1.0, c.ones.p);
    BEM_LAUNCH_CHECK();
    DevBuf<double> out;
    out.resize(N);
    const auto saved_apply = c.stats.n_apply, saved_apply_rhs = c.stats.n_apply_rhs;
    cudaEvent_t e0, e1;
    BEM_CUDA(cudaEventCreate(&e0));
    BEM_CUDA(cudaEventCreate(&e1));
    auto time_product = [&](int reps) {
        double f = 1.0, g = 0.0;
        const double *xl[1] = {c.ones.p};
        const double *xm[1] = {nullptr};
        double *o[1] = {out.p};
        offdiag_apply(c, 1, &f, xl, &g, xm, o, c.prm.precision);  // warm-up (chunk tables, buffers)
        BEM_CUDA(cudaEventRecord(e0, c.stream));
        for (int r = 0; r < reps; ++r) offdiag_apply(c, 1, &f, xl, &g, xm, o, c.prm.precision);
        BEM_CUDA(cudaEventRecord(e1, c.stream));
        BEM_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        BEM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        return ms / reps;
    };
    // 1. depth, with the default tiles
    c.tuned_stages = c.prm.m2l_stages;
    c.tuned_p2p_blocks = c.prm.p2p_blocks_per_sm > 0 ? c.prm.p2p_blocks_per_sm : 0;
    c.tuned_overlap = c.prm.overlap < 0 ? 1 : c.prm.overlap;
    const int saved_target = c.prm.leaf_target;
    c.prm.leaf_target = 64;
    c.level_override = 0;
    build_tree(c);
    c.prm.leaf_target = saved_target;
    const int L0 = c.tree.L;
    int best = L0;
    float best_ms = 0.f;
    for (int L = std::max(2, L0 - 1); L <= std::min(L0 + 1, c.tree.deep); ++L) {
        c.level_override = L;
        build_tree(c);
        c.m2l_chunks_h.clear();
        c.tc_chunks_ok[0] = c.tc_chunks_ok[1] = false;
        c.tm[0].ok = c.tm[1].ok = false;
        const float ms = time_product(1);
        if (L == std::max(2, L0 - 1) || ms < best_ms) {
            best = L;
            best_ms = ms;
        }
    }
    c.level_override = best;
    // 2. tiles at that depth
    std::vector<int> stages = {c.prm.m2l_stages};
    if (c.prm.m2l_stages == 0 && c.prm.precision == BEM_PREC_MIXED && c.prm.m2l_tensor_cores &&
        !c.prm.m2l_target_major)
        stages = {3, 2};
    std::vector<int> blocks = {c.tuned_p2p_blocks};
    if (c.prm.p2p_blocks_per_sm < 0 && c.prm.overlap) blocks = {0, 2, 4};
    std::vector<int> ovls = {c.tuned_overlap};
    if (c.prm.overlap < 0) ovls = {1, 2};
    if (stages.size() > 1 || blocks.size() > 1 || ovls.size() > 1) {
        build_tree(c);
        c.m2l_chunks_h.clear();
        c.tc_chunks_ok[0] = c.tc_chunks_ok[1] = false;
        c.tm[0].ok = c.tm[1].ok = false;
        float tbest = 0.f;
        int bs = stages[0], bb = blocks[0], bo = ovls[0];
        bool first = true;
        for (int ov : ovls)
            for (int st : stages)
                for (int bk : blocks) {
                    c.tuned_overlap = ov;
                    c.tuned_stages = st;
                    c.tuned_p2p_blocks = bk;
                    const float ms = time_product(3);
                    if (first || ms < tbest) {
                        tbest = ms;
                        bs = st;
                        bb = bk;
                        bo = ov;
                        first = false;
                    }
                }
        c.tuned_stages = bs;
        c.tuned_p2p_blocks = bb;
        c.tuned_overlap = bo;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c.level_override = 0;
    c.tuned_level = best;
    c.stats.n_apply = saved_apply;  // the timing products are not the caller's
    c.stats.n_apply_rhs = saved_apply_rhs;
}

void build_all(Context &c) {
    if (!c.mesh_ok) fail(BEM_ERR_NOT_BUILT, "no mesh uploaded");
    if (c.C > 1 && c.prm.mvp != BEM_MVP_FMM) fail(BEM_ERR_ARG, "independent clusters need the FMM product");
    cudaEvent_t e0, e1;
    BEM_CUDA(cudaEventCreate(&e0));
    BEM_CUDA(cudaEventCreate(&e1));
    BEM_CUDA(cudaEventRecord(e0, c.stream));
    c.built = false;
    const int64_t N = c.N;
    {
        // a non-finite coordinate (an uploaded NaN, or a time step that blew up) is reported as
        // such before any geometry or key is formed from it
        DevBuf<int> &badx = c.chk[0];
        badx.resize(1);
        BEM_CUDA(cudaMemsetAsync(badx.p, 0, sizeof(int), c.stream));
        k_check_finite<<<div_up(3 * N, 256), 256, 0, c.stream>>>(3 * N, c.xyz.p, badx.p);
        BEM_LAUNCH_CHECK();
        int hx = 0;
        BEM_CUDA(cudaMemcpyAsync(&hx, badx.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
        BEM_CUDA(cudaStreamSynchronize(c.stream));
        if (hx) fail(BEM_ERR_NAN, "non-finite vertex coordinate");
    }
    if (c.points_only) {  // unit weights, normals along z (unused: products use f only)
        c.s.resize(N);
        c.nrm.resize(3 * N);
        k_fill<<<div_up(N, 256), 256, 0, c.stream>>>(N, 1.0, c.s.p);
        k_fill<<<div_up(2 * N, 256), 256, 0, c.stream>>>(2 * N, 0.0, c.nrm.p);
        k_fill<<<div_up(N, 256), 256, 0, c.stream>>>(N, 1.0, c.nrm.p + 2 * N);
        BEM_LAUNCH_CHECK();
    } else {
        PhaseScope ps(c, PH_GEOMETRY);
        compute_vertex_geometry(c);
    }
    if (c.prm.mvp == BEM_MVP_FMM) {
        build_operators(c, c.ops, c.prm.p_fmm);
        if (c.prm.m2l_tensor_cores && m2l_tc_supported(c.ops.P) && c.ops.tc_Npad == 0) build_tc_tables(c, c.ops);
        c.tc_chunks_ok[0] = c.tc_chunks_ok[1] = false;
        c.tm[0].ok = c.tm[1].ok = false;
        c.tc_err.resize(1);
        BEM_CUDA(cudaMemsetAsync(c.tc_err.p, 0, sizeof(int), c.stream));
        if (c.prm.leaf_target == 0 && c.prm.fixed_level == 0 && c.tuned_level == 0) tune_tiles(c);
        c.level_override = c.prm.fixed_level == 0 ? c.tuned_level : 0;
        {
            PhaseScope ps(c, PH_TREE);
            build_tree(c);
        }
        c.m2l_chunks_h.clear();
        c.tc_chunks_ok[0] = c.tc_chunks_ok[1] = false;
        c.tm[0].ok = c.tm[1].ok = false;  // chunk tables follow the tree (the autotuner built others)
        c.stats.p2p_pairs = c.tree.p2p_pairs;
        c.stats.m2l_pairs = c.tree.n_m2l;
        c.stats.levels = c.tree.L;
        c.stats.leaves = c.tree.nb[c.tree.L];
        c.stats.m2l_stages = c.tuned_stages;
        c.stats.overlap = c.tuned_overlap;
        c.stats.p2p_blocks_per_sm = c.tuned_p2p_blocks;
        {
            const int P16 = (c.ops.P + 15) / 16 * 16;
            int64_t macs = 0;
            for (int k = 0; k < kNumM2LClasses; ++k) {
                const int64_t n = c.tree.m2l_class_off[k + 1] - c.tree.m2l_class_off[k];
                const int64_t K = c.ops.margin >= 0 ? std::min(P16, (c.ops.cls_p[k] * c.ops.cls_p[k] + 15) / 16 * 16)
                                                    : (int64_t)c.ops.P;
                macs += n * K * K;
            }
            c.stats.m2l_macs = macs;
        }
    } else {
        c.dir_hi.resize(3 * N);
        c.dir_lo.resize(3 * N);
        launch_split_hilo(3 * N, c.xyz.p, c.dir_hi.p, c.dir_lo.p, c.stream);
        c.stats.p2p_pairs = N * (N - 1);
        c.stats.m2l_pairs = 0;
        c.stats.levels = 0;
        c.stats.leaves = 0;
    }
    if (c.points_only) {  // no singular diagonal for point sources
        c.ldiag.resize(N);
        c.mdiag.resize(N);
        BEM_CUDA(cudaMemsetAsync(c.ldiag.p, 0, N * sizeof(double), c.stream));
        BEM_CUDA(cudaMemsetAsync(c.mdiag.p, 0, N * sizeof(double), c.stream));
        BEM_CUDA(cudaEventRecord(e1, c.stream));
        BEM_CUDA(cudaStreamSynchronize(c.stream));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        c.stats.last_build_ms = ms;
        c.built = true;
        return;
    }
    // diagonals from one 4-RHS off-diagonal product (Eqs. (s3), (s5))
    c.ones.resize(N);
    k_fill<<<div_up(N, 256), 256, 0, c.stream>>>(N, 1.0, c.ones.p);
    BEM_LAUNCH_CHECK();
    DevBuf<double> &tmp = c.diag_tmp;
    tmp.resize(4 * N);
    double fa[4] = {0.0, -1.0, -1.0, -1.0}, ga[4] = {1.0, 1.0, 1.0, 1.0};
    const double *xl[4] = {nullptr, c.nrm.p, c.nrm.p + N, c.nrm.p + 2 * N};
    const double *xm[4] = {c.ones.p, c.xyz.p, c.xyz.p + N, c.xyz.p + 2 * N};
    double *o[4] = {tmp.p, tmp.p + N, tmp.p + 2 * N, tmp.p + 3 * N};
    int dprec = c.prm.diag_precision < 0 ? c.prm.precision : c.prm.diag_precision;
    const Operators *dops = nullptr;
    if (c.prm.mvp == BEM_MVP_FMM) {
        const int dp = c.prm.diag_p_fmm > 0 ? c.prm.diag_p_fmm : std::min(c.prm.p_fmm + 2, kMaxPfmm);
        // tensor cores for the diagonal product: always in mode 2; in mode 3 (automatic) only while
        // every bubble has at most kDiagTcMaxVerts vertices. The identities cancel O(1) sums down
        // to O(h), so the far field's rounding is magnified by about R/h: on a 40962-vertex
        // bubble the BF16 split doubled the product error at p = 14, on 642-vertex bubbles it
        // left it unchanged.
        int64_t maxv = 0;
        for (size_t b = 0; b + 1 < c.vert_off.size(); ++b) maxv = std::max(maxv, c.vert_off[b + 1] - c.vert_off[b]);
        c.diag_tc = c.prm.m2l_tensor_cores == 2 || (c.prm.m2l_tensor_cores == 3 && maxv <= kDiagTcMaxVerts);
        if (dp != c.prm.p_fmm) {
            build_operators(c, c.ops_diag, dp);
            dops = &c.ops_diag;
            if (c.diag_tc && m2l_tc_supported(c.ops_diag.P) && c.ops_diag.tc_Npad == 0) build_tc_tables(c, c.ops_diag);
        }
    }
    offdiag_apply(c, 4, fa, xl, ga, xm, o, dprec, dops);
    c.ldiag.resize(N);
    c.mdiag.resize(N);
    PhaseScope ps(c, PH_DIAG);
    k_diag_identities<<<div_up(N, 256), 256, 0, c.stream>>>(N, o[0], o[1], o[2], o[3], c.xyz.p, c.nrm.p, c.ldiag.p,
                                                            c.mdiag.p);
    BEM_LAUNCH_CHECK();
    DevBuf<int> &bad = c.chk[1];
    bad.resize(1);
    BEM_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), c.stream));
    k_check_finite<<<div_up(N, 256), 256, 0, c.stream>>>(N, c.ldiag.p, bad.p);
    k_check_finite<<<div_up(N, 256), 256, 0, c.stream>>>(N, c.mdiag.p, bad.p);
    BEM_LAUNCH_CHECK();
    BEM_CUDA(cudaEventRecord(e1, c.stream));
    int hb = 0;
    BEM_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    BEM_CUDA(cudaStreamSynchronize(c.stream));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c.stats.last_build_ms = ms;
    if (hb) fail(BEM_ERR_NAN, "non-finite singular diagonal");
    if (c.prm.mvp == BEM_MVP_FMM) {
        int he = 0;
        BEM_CUDA(cudaMemcpy(&he, c.tc_err.p, sizeof(int), cudaMemcpyDeviceToHost));
        if (he) fail(BEM_ERR_TIMEOUT, "tensor-core M2L wait ran out");
    }
    c.built = true;
}

// b = -phi/2 + M phi, then GMRES from q (device pointers).
void solve_internal(Context &c, const double *phi, double *q, int *it, double *rr) {
    c.bv.resize(c.N);
    apply_full(c, 0.0, nullptr, 1.0, phi, c.bv.p);
    k_rhs_combine<<<div_up(c.N, 256), 256, 0, c.stream>>>(c.N, phi, c.bv.p);
    BEM_LAUNCH_CHECK();
    if (c.C > 1) gmres_solve_batched(c, c.bv.p, q, it, rr);
    else gmres_solve(c, c.bv.p, q, it, rr);
}

}  // namespace bem

using namespace bem;

extern "C" {

int bem_params_default(bem_params *p) {
    if (!p) return BEM_ERR_ARG;
    std::memset(p, 0, sizeof(*p));
    p->p_fmm = 14;
    p->leaf_target = 64;
    p->fixed_level = 0;
    p->precision = BEM_PREC_MIXED;
    p->mvp = BEM_MVP_FMM;
    p->diag_precision = -1;
    p->diag_p_fmm = -1;
    p->overlap = -1;
    p->m2l_tensor_cores = 3;
    p->gmres_precond = 0;
    p->gmres_maxit = 100;
    p->gmres_restart = 0;
    p->gmres_tol = 1e-6;
    p->m2l_stages = 0;
    p->p2p_blocks_per_sm = -1;
    p->m2l_order_margin = 6;
    p->m2l_target_major = 1;
    return BEM_OK;
}

int bem_create(void **ctx_out, const bem_params *p, void *stream) {
    if (!ctx_out) return BEM_ERR_ARG;
    *ctx_out = nullptr;
    Context *c = nullptr;
    try {
        bem_params prm;
        if (p) prm = *p;
        else bem_params_default(&prm);
        check_params(prm);
        c = new Context();
        c->prm = prm;
        c->stream = static_cast<cudaStream_t>(stream);
        BEM_CUDA(cudaGetDevice(&c->device));
        BEM_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
        c->tuned_stages = prm.m2l_stages;
        c->tuned_p2p_blocks = prm.p2p_blocks_per_sm < 0 ? 0 : prm.p2p_blocks_per_sm;
        c->tuned_overlap = prm.overlap < 0 ? 1 : prm.overlap;
        *ctx_out = c;
        return BEM_OK;
    } catch (const Error &e) {
        g_create_error = e.msg;
        delete c;
        return e.code;
    }
}

void bem_destroy(void *ctx) {
    if (!ctx) return;
    Context *c = static_cast<Context *>(ctx);
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    delete c;
}

int bem_set_stream(void *ctx, void *stream) {
    return guarded(ctx, [&](Context &c) { c.stream = static_cast<cudaStream_t>(stream); });
}

const char *bem_last_error(const void *ctx) {
    if (!ctx) return g_create_error.c_str();
    return static_cast<const Context *>(ctx)->err.c_str();
}

int bem_mesh_upload(void *ctx, int64_t N, const double *xyz, int64_t T, const int32_t *tri, int64_t M,
                    const int64_t *vert_off, const int64_t *tri_off) {
    return guarded(ctx, [&](Context &c) {
        if (N < 2 || T < 1 || M < 1 || !xyz || !tri || !vert_off || !tri_off) fail(BEM_ERR_ARG, "bad mesh sizes or null arrays");
        if (N > (int64_t)INT32_MAX / 2 || T > (int64_t)INT32_MAX / 3) fail(BEM_ERR_ARG, "mesh too large for 32-bit indices");
        c.built = false;
        c.mesh_ok = false;
        c.points_only = false;
        c.bp.ready = false;
        c.tuned_level = 0;
        c.C = 1;
        c.cluster_boff.clear();
        c.N = N;
        c.T = T;
        c.M = M;
        c.xyz.resize(3 * N);
        c.tri.resize(3 * T);
        auto kind = [&](const void *p) { return is_device_ptr(c, p) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; };
        BEM_CUDA(cudaMemcpyAsync(c.xyz.p, xyz, 3 * N * sizeof(double), kind(xyz), c.stream));
        BEM_CUDA(cudaMemcpyAsync(c.tri.p, tri, 3 * T * sizeof(int32_t), kind(tri), c.stream));
        c.vert_off.resize(M + 1);
        c.tri_off.resize(M + 1);
        auto kind_h = [&](const void *p) { return is_device_ptr(c, p) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost; };
        BEM_CUDA(cudaMemcpyAsync(c.vert_off.data(), vert_off, (M + 1) * sizeof(int64_t), kind_h(vert_off), c.stream));
        BEM_CUDA(cudaMemcpyAsync(c.tri_off.data(), tri_off, (M + 1) * sizeof(int64_t), kind_h(tri_off), c.stream));
        BEM_CUDA(cudaStreamSynchronize(c.stream));
        if (c.vert_off[0] != 0 || c.vert_off[M] != N || c.tri_off[0] != 0 || c.tri_off[M] != T)
            fail(BEM_ERR_ARG, "offsets must start at 0 and end at N / T");
        for (int64_t m = 0; m < M; ++m)
            if (c.vert_off[m + 1] < c.vert_off[m] || c.tri_off[m + 1] < c.tri_off[m])
                fail(BEM_ERR_ARG, "offsets must be non-decreasing");
        c.voff_d.resize(M + 1);
        BEM_CUDA(cudaMemcpyAsync(c.voff_d.p, c.vert_off.data(), (M + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                                 c.stream));
        build_vertex_triangle_csr(c);
        c.mesh_ok = true;
    });
}

__global__ void k_fill_cluster(const int64_t *__restrict__ cvoff, int32_t *__restrict__ vcid) {
    const int c = blockIdx.x;
    for (int64_t i = cvoff[c] + threadIdx.x; i < cvoff[c + 1]; i += blockDim.x) vcid[i] = c;
}

int bem_mesh_set_clusters(void *ctx, int64_t C, const int64_t *bubble_off) {
    return guarded(ctx, [&](Context &c) {
        if (!c.mesh_ok || c.points_only) fail(BEM_ERR_NOT_BUILT, "upload a mesh first");
        if (C < 1 || C > 256 || !bubble_off) fail(BEM_ERR_ARG, "cluster count must be in 1..256");
        std::vector<int64_t> bo(C + 1);
        auto k = is_device_ptr(c, bubble_off) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
        BEM_CUDA(cudaMemcpy(bo.data(), bubble_off, (C + 1) * sizeof(int64_t), k));
        if (bo[0] != 0 || bo[C] != c.M) fail(BEM_ERR_ARG, "bubble offsets must start at 0 and end at M");
        for (int64_t i = 0; i < C; ++i)
            if (bo[i + 1] <= bo[i]) fail(BEM_ERR_ARG, "every cluster needs at least one bubble");
        c.built = false;
        c.C = C;
        c.cluster_boff = bo;
        if (C > 1) {
            std::vector<int64_t> cv(C + 1);
            for (int64_t i = 0; i <= C; ++i) cv[i] = c.vert_off[bo[i]];
            DevBuf<int64_t> dcv;
            dcv.resize(C + 1);
            BEM_CUDA(cudaMemcpyAsync(dcv.p, cv.data(), (C + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c.stream));
            c.vcid.resize(c.N);
            k_fill_cluster<<<(unsigned)C, 256, 0, c.stream>>>(dcv.p, c.vcid.p);
            BEM_LAUNCH_CHECK();
            BEM_CUDA(cudaStreamSynchronize(c.stream));
        }
    });
}

int bem_points_upload(void *ctx, int64_t N, const double *xyz) {
    return guarded(ctx, [&](Context &c) {
        if (N < 2 || !xyz) fail(BEM_ERR_ARG, "bad point count or null array");
        if (N > (int64_t)INT32_MAX / 2) fail(BEM_ERR_ARG, "too many points for 32-bit indices");
        c.built = false;
        c.mesh_ok = false;
        c.points_only = true;
        c.bp.ready = false;
        c.tuned_level = 0;
        c.C = 1;
        c.cluster_boff.clear();
        c.N = N;
        c.T = 0;
        c.M = 1;
        c.xyz.resize(3 * N);
        auto k = is_device_ptr(c, xyz) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        BEM_CUDA(cudaMemcpyAsync(c.xyz.p, xyz, 3 * N * sizeof(double), k, c.stream));
        c.vert_off = {0, N};
        c.tri_off = {0, 0};
        BEM_CUDA(cudaStreamSynchronize(c.stream));
        c.mesh_ok = true;
    });
}

int bem_mesh_update_xyz(void *ctx, const double *xyz) {
    return guarded(ctx, [&](Context &c) {
        if (!c.mesh_ok) fail(BEM_ERR_NOT_BUILT, "no mesh uploaded");
        if (!xyz) fail(BEM_ERR_ARG, "null xyz");
        c.built = false;
        auto k = is_device_ptr(c, xyz) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        BEM_CUDA(cudaMemcpyAsync(c.xyz.p, xyz, 3 * c.N * sizeof(double), k, c.stream));
    });
}

int fmm_build(void *ctx) {
    return guarded(ctx, [&](Context &c) { build_all(c); });
}

int bem_apply(void *ctx, double f, const double *xL, double g, const double *xM, double *out) {
    return guarded(ctx, [&](Context &c) {
        require_built(c);
        if ((f != 0.0 && !xL) || (g != 0.0 && !xM)) fail(BEM_ERR_ARG, "null input with a non-zero coefficient");
        const double *dl = f != 0.0 ? dev_in(c, xL, c.N, 0) : nullptr;
        const double *dm = g != 0.0 ? dev_in(c, xM, c.N, 1) : nullptr;
        OutView ov(c, out, c.N);
        apply_full(c, f, dl, g, dm, ov.dev);
        ov.finish();
    });
}

int bem_apply_sl(void *ctx, const double *q, double *out) { return bem_apply(ctx, 1.0, q, 0.0, nullptr, out); }

int bem_apply_dl(void *ctx, const double *phi, double *out) { return bem_apply(ctx, 0.0, nullptr, 1.0, phi, out); }

int bem_rhs(void *ctx, const double *phi, double *b) {
    return guarded(ctx, [&](Context &c) {
        require_built(c);
        if (!phi) fail(BEM_ERR_ARG, "null phi");
        const double *dp = dev_in(c, phi, c.N, 0);
        OutView ov(c, b, c.N);
        apply_full(c, 0.0, nullptr, 1.0, dp, ov.dev);
        k_rhs_combine<<<div_up(c.N, 256), 256, 0, c.stream>>>(c.N, dp, ov.dev);
        BEM_LAUNCH_CHECK();
        ov.finish();
    });
}

int bem_precond_apply(void *ctx, const double *y, double *z) {
    return guarded(ctx, [&](Context &c) {
        require_built(c);
        if (!y || !z) fail(BEM_ERR_ARG, "null y or z");
        const double *dy = dev_in(c, y, c.N, 0);
        OutView ov(c, z, c.N);
        block_precond_prepare(c);
        block_precond_apply(c, dy, ov.dev);
        ov.finish();
        block_precond_check(c);
    });
}

int bem_solve(void *ctx, const double *phi, double *q_inout, int32_t *iters, double *relres) {
    int it = 0;
    double rr = 0.0;
    int rc = guarded(ctx, [&](Context &c) {
        require_built(c);
        if (!phi || !q_inout) fail(BEM_ERR_ARG, "null phi or q");
        const double *dp = dev_in(c, phi, c.N, 0);
        const bool host_q = !is_device_ptr(c, q_inout);
        double *dq = q_inout;
        if (host_q) {
            c.stage_in[1].resize(c.N);
            dq = c.stage_in[1].p;
            BEM_CUDA(cudaMemcpyAsync(dq, q_inout, c.N * sizeof(double), cudaMemcpyHostToDevice, c.stream));
        }
        struct CopyBack {
            Context &c;
            bool host;
            double *user, *dev;
            ~CopyBack() {
                if (host) {
                    cudaMemcpyAsync(user, dev, c.N * sizeof(double), cudaMemcpyDeviceToHost, c.stream);
                    cudaStreamSynchronize(c.stream);
                }
            }
        } cb{c, host_q, q_inout, dq};
        solve_internal(c, dp, dq, &it, &rr);
    });
    if (iters) *iters = it;
    if (relres) *relres = rr;
    if (rc == BEM_ERR_NOCONV && ctx) {
        Context *c = static_cast<Context *>(ctx);
        if (iters) *iters = c->stats.last_iters;
        if (relres) *relres = c->stats.last_relres;
    }
    return rc;
}

int bem_get_geometry(void *ctx, double *s, double *n, double *ldiag, double *mdiag) {
    return guarded(ctx, [&](Context &c) {
        require_built(c);
        struct Item {
            double *dst;
            const double *src;
            int64_t n;
        } items[4] = {{s, c.s.p, c.N}, {n, c.nrm.p, 3 * c.N}, {ldiag, c.ldiag.p, c.N}, {mdiag, c.mdiag.p, c.N}};
        for (auto &it : items) {
            if (!it.dst) continue;
            auto k = is_device_ptr(c, it.dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
            BEM_CUDA(cudaMemcpyAsync(it.dst, it.src, it.n * sizeof(double), k, c.stream));
        }
        BEM_CUDA(cudaStreamSynchronize(c.stream));
    });
}

int bem_step_params_default(bem_step_params *sp) {
    if (!sp) return BEM_ERR_ARG;
    std::memset(sp, 0, sizeof(*sp));
    sp->sigma = 0.073;
    sp->kappa = 1.4;
    sp->pa = 1.0;
    sp->omega = 1.2566370614359172;
    sp->courant = 0.1;
    sp->dt = 0.0;
    sp->pf = 6;
    sp->guess = 2;
    sp->ab_order = 6;
    sp->corrector = 0;
    sp->rk_order = 4;
    return BEM_OK;
}

int bem_step_init(void *ctx, const double *phi0, const double *q0, const bem_step_params *sp) {
    return guarded(ctx, [&](Context &c) {
        if (!phi0) fail(BEM_ERR_ARG, "null phi0");
        bem_step_params p;
        if (sp) p = *sp;
        else bem_step_params_default(&p);
        const double *dp = dev_in(c, phi0, c.N, 0);
        const double *dq = q0 ? dev_in(c, q0, c.N, 1) : nullptr;
        step_init(c, dp, dq, p);
    });
}

int bem_step(void *ctx, bem_step_stats *st) {
    return guarded(ctx, [&](Context &c) {
        bem_step_stats s{};
        step_advance(c, s);
        if (st) *st = s;
    });
}

int bem_step_get_state(void *ctx, double *xyz, double *phi, double *q, double *t) {
    return guarded(ctx, [&](Context &c) { step_get_state(c, xyz, phi, q, t); });
}

int bem_step_set_state(void *ctx, const double *xyz, const double *phi, const double *q) {
    return guarded(ctx, [&](Context &c) { step_set_state(c, xyz, phi, q); });
}

int bem_step_filter(void *ctx, const double *x, double *y) {
    return guarded(ctx, [&](Context &c) { step_filter(c, x, y); });
}

int bem_step_save(void *ctx, void *buf, int64_t cap, int64_t *size) {
    return guarded(ctx, [&](Context &c) {
        if (!c.mesh_ok) fail(BEM_ERR_NOT_BUILT, "no mesh uploaded");
        const int64_t need = step_checkpoint_size(c);
        if (size) *size = need;
        if (buf) step_save(c, buf, cap);
    });
}

int bem_step_load(void *ctx, const void *buf, int64_t size) {
    return guarded(ctx, [&](Context &c) {
        if (!buf) fail(BEM_ERR_ARG, "null checkpoint");
        step_load(c, buf, size);
    });
}

int bem_mlp_init(void *ctx, int32_t hidden, int32_t lmax, uint64_t seed) {
    return guarded(ctx, [&](Context &c) { mlp_init(c, hidden, lmax, seed, step_initial_xyz(c)); });
}

int bem_mlp_set_mode(void *ctx, int32_t record, int32_t use_guess, int32_t compare) {
    return guarded(ctx, [&](Context &c) { mlp_set_mode(c, record, use_guess, compare); });
}

int bem_mlp_train(void *ctx, int32_t epochs, int32_t batch, double lr, double *last_loss) {
    return guarded(ctx, [&](Context &c) {
        if (epochs < 1 || batch < 1 || !(lr > 0.0)) fail(BEM_ERR_ARG, "epochs, batch and lr must be positive");
        double l = mlp_train(c, epochs, batch, lr);
        if (last_loss) *last_loss = l;
    });
}

int bem_mlp_loss_grad(void *ctx, int32_t B, const double *F, const double *T, double *loss, double *grads) {
    return guarded(ctx, [&](Context &c) {
        if (B < 1 || !F || !T || !grads) fail(BEM_ERR_ARG, "bad batch or null array");
        const int *d = mlp_dims(c);
        const double *dF = dev_in(c, F, (int64_t)B * d[0], 0);
        const double *dT = dev_in(c, T, (int64_t)B * d[4], 1);
        int64_t np = mlp_num_params(*c.mlp);
        OutView ov(c, grads, np);
        double l = mlp_loss_grad(c, B, dF, dT, ov.dev);
        ov.finish();
        if (loss) *loss = l;
    });
}

int bem_mlp_forward(void *ctx, int32_t B, const double *F, double *Y) {
    return guarded(ctx, [&](Context &c) {
        if (B < 1 || !F || !Y) fail(BEM_ERR_ARG, "bad batch or null array");
        const int *d = mlp_dims(c);
        const double *dF = dev_in(c, F, (int64_t)B * d[0], 0);
        OutView ov(c, Y, (int64_t)B * d[4]);
        mlp_forward(c, B, dF, ov.dev);
        ov.finish();
    });
}

int bem_mlp_get_params(void *ctx, double *out) {
    return guarded(ctx, [&](Context &c) {
        if (!out) fail(BEM_ERR_ARG, "null output");
        std::vector<double> h(mlp_num_params(*c.mlp));
        mlp_get_params(c, h.data());
        auto k = is_device_ptr(c, out) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
        BEM_CUDA(cudaMemcpy(out, h.data(), h.size() * sizeof(double), k));
    });
}

int bem_mlp_set_params(void *ctx, const double *in) {
    return guarded(ctx, [&](Context &c) {
        if (!in) fail(BEM_ERR_ARG, "null input");
        std::vector<double> h(mlp_num_params(*c.mlp));
        auto k = is_device_ptr(c, in) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
        BEM_CUDA(cudaMemcpy(h.data(), in, h.size() * sizeof(double), k));
        mlp_set_params(c, h.data());
    });
}

int bem_mlp_info(void *ctx, bem_mlp_summary *out) {
    return guarded(ctx, [&](Context &c) {
        if (!out) fail(BEM_ERR_ARG, "null output");
        if (!c.mlp) fail(BEM_ERR_NOT_BUILT, "bem_mlp_init has not been called");
        const int *d = mlp_dims(c);
        for (int i = 0; i < 5; ++i) out->dims[i] = d[i];
        out->reserved = 0;
        out->num_params = mlp_num_params(*c.mlp);
        out->samples = mlp_samples(c);
        const MlpStats &ms = mlp_stats(c);
        out->compared_solves = ms.solves;
        out->iters_guess = ms.iters_guess;
        out->iters_fallback = ms.iters_fallback;
        out->res0_guess = ms.res0_guess;
        out->res0_fallback = ms.res0_fallback;
    });
}

int bem_get_residual_history(void *ctx, double *out, int32_t max, int32_t *count) {
    return guarded(ctx, [&](Context &c) {
        int n = (int)c.res_hist.size();
        if (count) *count = n;
        if (out)
            for (int i = 0; i < n && i < max; ++i) out[i] = c.res_hist[i];
    });
}

int bem_get_stats(void *ctx, bem_stats *out) {
    return guarded(ctx, [&](Context &c) {
        if (!out) fail(BEM_ERR_ARG, "null stats");
        c.stats.n_launches = g_launch_count;
        *out = c.stats;
    });
}

int bem_profile_enable(void *ctx, int on) {
    return guarded(ctx, [&](Context &c) {
        BEM_CUDA(cudaStreamSynchronize(c.stream));
        for (auto &r : c.prof.recs) {
            c.prof.pool.push_back(r.a);
            c.prof.pool.push_back(r.b);
        }
        c.prof.recs.clear();
        c.prof.on = on != 0;
    });
}

int bem_profile_read(void *ctx, double *ms, int64_t *intervals) {
    return guarded(ctx, [&](Context &c) {
        BEM_CUDA(cudaStreamSynchronize(c.stream));
        double acc[PH_COUNT] = {0};
        int64_t cnt[PH_COUNT] = {0};
        for (auto &r : c.prof.recs) {
            float t = 0.f;
            BEM_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
            acc[r.phase] += t;
            cnt[r.phase] += 1;
            c.prof.pool.push_back(r.a);
            c.prof.pool.push_back(r.b);
        }
        c.prof.recs.clear();
        for (int i = 0; i < PH_COUNT; ++i) {
            if (ms) ms[i] = acc[i];
            if (intervals) intervals[i] = cnt[i];
        }
    });
}

const char *bem_phase_name(int i) {
    static const char *names[PH_COUNT] = {"geometry", "tree", "operators", "strengths", "p2m", "m2m", "m2l",
                                          "l2l", "l2p", "p2p", "direct", "diag", "gmres", "m2l_reduce", "m2l_cc"};
    return (i >= 0 && i < PH_COUNT) ? names[i] : nullptr;
}

int bem_get_cluster_stats(void *ctx, int64_t C, int32_t *iters, double *relres, double *done_ms, double *solve_ms) {
    return guarded(ctx, [&](Context &c) {
        if (C != c.C) fail(BEM_ERR_ARG, "C must equal the context's cluster count");
        if (c.cl_iters.size() != (size_t)C) fail(BEM_ERR_NOT_BUILT, "no clustered solve has run");
        for (int64_t k = 0; k < C; ++k) {
            if (iters) iters[k] = c.cl_iters[k];
            if (relres) relres[k] = c.cl_relres[k];
            if (done_ms) done_ms[k] = c.cl_done_ms[k];
        }
        if (solve_ms) *solve_ms = c.cl_solve_ms;
    });
}

int bem_m2l_orders(int32_t p_fmm, int32_t margin, int32_t *orders) {
    if (!orders || p_fmm < 2 || p_fmm > kMaxPfmm || margin < -1) return BEM_ERR_ARG;
    const std::vector<int> o = m2l_class_orders(p_fmm, margin);
    for (int k = 0; k < kNumM2LClasses; ++k) orders[k] = o[k];
    return BEM_OK;
}

int bem_reset_stats(void *ctx) {
    return guarded(ctx, [&](Context &c) {
        c.stats.n_apply = 0;
        c.stats.n_apply_rhs = 0;
    });
}

}  // extern "C"
