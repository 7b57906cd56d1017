// GMRES for independent clusters stepped together (bem_mesh_set_clusters), Section 3.8 applied
// to every cluster's own system. The operator of C independent clusters is block diagonal
// (no interaction crosses clusters), so the C systems are solved as C GMRES processes in
// lockstep: one operator product per iteration serves all clusters (the products, the
// preconditioner and the vector updates are one launch each for all of them), while the
// Arnoldi inner products, norms, Hessenberg matrices, Givens rotations, residual estimates,
// convergence decisions and solution updates are per cluster. A cluster stops when its own
// relative residual |b_c - A_c x_c| / |b_c| meets the tolerance: its solution is updated at the
// iteration it converges (its later basis vectors are zero, so further products leave it
// unchanged), and the solve ends when every cluster has converged. A single Krylov space over
// the stacked system would stop on the global residual, which leaves clusters with small
// right-hand sides short of their own tolerance.
//
// All reductions run over fixed segments of at most kSeg vertices of one cluster and are
// combined per cluster in a fixed order, so a solve is reproducible run to run.
#include "internal.h"

#include <algorithm>
#include <cmath>

namespace bem {
namespace {

constexpr int SEG_THREADS = 256;
constexpr int64_t kSeg = 16384;  // vertices per reduction segment
constexpr int SEG_JB = 8;        // basis vectors per pass over w

// partial[j * nseg + s] = sum over segment s of V_j . w
__global__ void __launch_bounds__(SEG_THREADS) k_segdot(int nv, int nseg, const int64_t *__restrict__ s0,
                                                       const int64_t *__restrict__ s1, const double *__restrict__ V,
                                                       size_t ldv, const double *__restrict__ w,
                                                       double *__restrict__ partial) {
    __shared__ double red[SEG_THREADS / 32][SEG_JB];
    const int s = blockIdx.x;
    const int64_t i0 = s0[s], i1 = s1[s];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j0 = 0; j0 < nv; j0 += SEG_JB) {
        const int nj = min(SEG_JB, nv - j0);
        double acc[SEG_JB];
#pragma unroll
        for (int jj = 0; jj < SEG_JB; ++jj) acc[jj] = 0.0;
        for (int64_t i = i0 + threadIdx.x; i < i1; i += SEG_THREADS) {
            const double wi = w[i];
#pragma unroll
            for (int jj = 0; jj < SEG_JB; ++jj)
                if (jj < nj) acc[jj] = fma(V[(size_t)(j0 + jj) * ldv + i], wi, acc[jj]);
        }
#pragma unroll
        for (int jj = 0; jj < SEG_JB; ++jj) {
            double t = acc[jj];
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) red[warp][jj] = t;
        }
        __syncthreads();
        if (threadIdx.x < nj) {
            double t = 0.0;
            for (int k = 0; k < SEG_THREADS / 32; ++k) t += red[k][threadIdx.x];
            partial[(size_t)(j0 + threadIdx.x) * nseg + s] = t;
        }
        __syncthreads();
    }
}

// out[j * C + c] = (accumulate ? out : 0) + sum of the cluster's segments in order
__global__ void k_segfinal(int nv, int C, int nseg, const int32_t *__restrict__ seg_off,
                           const double *__restrict__ partial, double *__restrict__ out, int accumulate) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nv * C) return;
    const int j = e / C, c = e % C;
    double t = 0.0;
    for (int s = seg_off[c]; s < seg_off[c + 1]; ++s) t += partial[(size_t)j * nseg + s];
    out[e] = (accumulate ? out[e] : 0.0) + t;
}

// w[i] += sign * sum_j h[j * C + cl(i)] V_j[i]
__global__ void k_segaxpy(int nv, int64_t N, int C, const double *__restrict__ V, size_t ldv,
                          const double *__restrict__ h, const int32_t *__restrict__ cl, double sign,
                          double *__restrict__ w) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = cl[i];
        double acc = 0.0;
        for (int j = 0; j < nv; ++j) acc = fma(h[(size_t)j * C + c], V[j * ldv + i], acc);
        w[i] += sign * acc;
    }
}

// v = w / |w|_c for active clusters, 0 otherwise; norms from nrm2[c]
__global__ void k_segnormalise(int64_t N, const double *__restrict__ w, const double *__restrict__ nrm2,
                               const int32_t *__restrict__ cl, const int32_t *__restrict__ active,
                               double *__restrict__ v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = cl[i];
        const double nn = sqrt(fmax(nrm2[c], 0.0));
        v[i] = (active[c] && nn > 0.0) ? w[i] / nn : 0.0;
    }
}

// y = alpha x + beta y
__global__ void k_axpby_b(int64_t N, double alpha, const double *__restrict__ x, double beta, double *__restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = alpha * x[i] + beta * y[i];
}

// Per cluster (one thread each): column k of its Hessenberg matrix from h[j * C + c] (j <= k)
// and |w| (nrm2), through its previous rotations, a new rotation, the rotated right-hand side,
// and res[c] = |g_{k+1}|. Inactive clusters are left unchanged.
__global__ void k_givens_b(int k, int m, int C, const double *__restrict__ h, const double *__restrict__ nrm2,
                           const int32_t *__restrict__ active, double *__restrict__ H, double *__restrict__ cs,
                           double *__restrict__ sn, double *__restrict__ g, double *__restrict__ res) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C || !active[c]) return;
    double *Hc = H + (size_t)c * (m + 1) * m;
    double *col = Hc + (size_t)k * (m + 1);
    double *csc = cs + (size_t)c * (m + 1), *snc = sn + (size_t)c * (m + 1), *gc = g + (size_t)c * (m + 2);
    for (int i = 0; i <= k; ++i) col[i] = h[(size_t)i * C + c];
    col[k + 1] = sqrt(fmax(nrm2[c], 0.0));
    for (int j = 0; j < k; ++j) {
        const double t = csc[j] * col[j] + snc[j] * col[j + 1];
        col[j + 1] = -snc[j] * col[j] + csc[j] * col[j + 1];
        col[j] = t;
    }
    const double d = hypot(col[k], col[k + 1]);
    double cc = 1.0, ss = 0.0;
    if (d != 0.0) {
        cc = col[k] / d;
        ss = col[k + 1] / d;
    }
    csc[k] = cc;
    snc[k] = ss;
    col[k] = d;
    col[k + 1] = 0.0;
    gc[k + 1] = -ss * gc[k];
    gc[k] = cc * gc[k];
    res[c] = fabs(gc[k + 1]);
}

// Per cluster: g = (beta_c, 0, ...) at a cycle start
__global__ void k_cycle_start_b(int m, int C, const double *__restrict__ beta2, double *__restrict__ g) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    double *gc = g + (size_t)c * (m + 2);
    gc[0] = sqrt(fmax(beta2[c], 0.0));
    for (int i = 1; i < m + 2; ++i) gc[i] = 0.0;
}

// Per cluster in `sel`: back substitution H(0:kk,0:kk) y = g(0:kk) into y[j * C + c]; the
// other clusters get y = 0 (their solutions are left unchanged by the update that follows).
__global__ void k_backsolve_b(int m, int C, const int32_t *__restrict__ kk, const int32_t *__restrict__ sel,
                              const double *__restrict__ H, const double *__restrict__ g, double *__restrict__ y) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const int n = sel[c] ? kk[c] : 0;
    const double *Hc = H + (size_t)c * (m + 1) * m;
    const double *gc = g + (size_t)c * (m + 2);
    for (int j = m - 1; j >= n; --j) y[(size_t)j * C + c] = 0.0;
    for (int i = n - 1; i >= 0; --i) {
        double s = gc[i];
        for (int j = i + 1; j < n; ++j) s -= Hc[(size_t)j * (m + 1) + i] * y[(size_t)j * C + c];
        const double d = Hc[(size_t)i * (m + 1) + i];
        y[(size_t)i * C + c] = d != 0.0 ? s / d : 0.0;
    }
}

// z = y / d (right Jacobi preconditioning)
__global__ void k_jacobi_b(int64_t N, const double *__restrict__ d, const double *__restrict__ y, double *__restrict__ z) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        z[i] = y[i] / d[i];
}

// x[i] = 0 where the cluster of i is flagged
__global__ void k_zero_clusters(int64_t N, const int32_t *__restrict__ cl, const int32_t *__restrict__ flag,
                                double *__restrict__ x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        if (flag[cl[i]]) x[i] = 0.0;
}

int grid_b(int64_t N) { return (int)std::min<int64_t>(div_up(N, 256), 152 * 8); }

}  // namespace

void gmres_solve_batched(Context &c, const double *b, double *x, int *iters_out, double *relres_out) {
    const int64_t N = c.N;
    const int C = (int)c.C;
    const int maxit = std::max(1, c.prm.gmres_maxit);
    const int m = std::min({maxit, c.prm.gmres_restart > 0 ? c.prm.gmres_restart : maxit, 127});
    const double tol = c.prm.gmres_tol;
    const int pmode = c.prm.gmres_precond;
    auto &G = c.gb;
    // reduction segments: at most kSeg vertices of one cluster each
    if (G.C != C || G.N != N) {
        std::vector<int64_t> s0, s1;
        std::vector<int32_t> off(C + 1, 0);
        for (int k = 0; k < C; ++k) {
            const int64_t a = c.vert_off[c.cluster_boff[k]], e = c.vert_off[c.cluster_boff[k + 1]];
            for (int64_t i = a; i < e; i += kSeg) {
                s0.push_back(i);
                s1.push_back(std::min(e, i + kSeg));
            }
            off[k + 1] = (int32_t)s0.size();
        }
        G.nseg = (int)s0.size();
        G.s0.resize(G.nseg);
        G.s1.resize(G.nseg);
        G.seg_off.resize(C + 1);
        BEM_CUDA(cudaMemcpyAsync(G.s0.p, s0.data(), s0.size() * sizeof(int64_t), cudaMemcpyHostToDevice, c.stream));
        BEM_CUDA(cudaMemcpyAsync(G.s1.p, s1.data(), s1.size() * sizeof(int64_t), cudaMemcpyHostToDevice, c.stream));
        BEM_CUDA(cudaMemcpyAsync(G.seg_off.p, off.data(), off.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                 c.stream));
        G.C = C;
        G.N = N;
    }
    if (pmode != 0) c.zv.resize(N);
    if (pmode == 2) block_precond_prepare(c);
    c.V.resize((size_t)(m + 1) * N);
    c.wv.resize(N);
    c.rv.resize(N);
    G.partial.resize((size_t)(m + 2) * G.nseg);
    G.h.resize((size_t)(m + 2) * C);
    G.h2.resize((size_t)(m + 2) * C);
    G.H.resize((size_t)C * (m + 1) * m);
    G.cs.resize((size_t)C * (m + 1));
    G.sn.resize((size_t)C * (m + 1));
    G.g.resize((size_t)C * (m + 2));
    G.y.resize((size_t)m * C);
    G.nrm2.resize(C);
    G.res.resize(C);
    G.active.resize(C);
    G.sel.resize(C);
    G.kk.resize(C);
    double *hres = c.hscal.get(2 * (size_t)C);
    const int g1 = grid_b(N), gc = div_up(C, 128);

    // z = P y: Jacobi (y / L_ii) or the bubble blocks (both act within bubbles)
    auto precond_apply = [&](const double *yv, double *z) {
        PhaseScope ps(c, PH_GMRES);
        if (pmode == 1) {
            k_jacobi_b<<<g1, 256, 0, c.stream>>>(N, c.ldiag.p, yv, z);
            BEM_LAUNCH_CHECK();
        } else {
            block_precond_apply(c, yv, z);
        }
    };
    auto segdots = [&](int nv, const double *V, size_t ldv, const double *w, double *out, int acc) {
        PhaseScope ps(c, PH_GMRES);
        k_segdot<<<G.nseg, SEG_THREADS, 0, c.stream>>>(nv, G.nseg, G.s0.p, G.s1.p, V, ldv, w, G.partial.p);
        BEM_LAUNCH_CHECK();
        k_segfinal<<<div_up((int64_t)nv * C, 128), 128, 0, c.stream>>>(nv, C, G.nseg, G.seg_off.p, G.partial.p, out,
                                                                     acc);
        BEM_LAUNCH_CHECK();
    };
    auto read_C = [&](const double *dev) {
        BEM_CUDA(cudaMemcpyAsync(hres, dev, C * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
        BEM_CUDA(cudaStreamSynchronize(c.stream));
        return std::vector<double>(hres, hres + C);
    };
    auto upload = [&](DevBuf<int32_t> &dst, const std::vector<int32_t> &v) {
        BEM_CUDA(cudaMemcpyAsync(dst.p, v.data(), C * sizeof(int32_t), cudaMemcpyHostToDevice, c.stream));
        BEM_CUDA(cudaStreamSynchronize(c.stream));  // the host vector may change right after
    };
    // x += t and d += t, t = P V y for the clusters in `sel` (y is zero for the others); the work
    // vector w is free whenever this runs (after a Givens step, or at the end of a cycle)
    auto update = [&](const std::vector<int32_t> &kk, const std::vector<int32_t> &sel) {
        upload(G.kk, kk);
        upload(G.sel, sel);
        int kmax = 0;
        for (int k = 0; k < C; ++k)
            if (sel[k]) kmax = std::max(kmax, kk[k]);
        if (kmax == 0) return;
        PhaseScope ps(c, PH_GMRES);
        k_backsolve_b<<<gc, 128, 0, c.stream>>>(m, C, G.kk.p, G.sel.p, G.H.p, G.g.p, G.y.p);
        BEM_LAUNCH_CHECK();
        if (pmode == 0) {
            BEM_CUDA(cudaMemsetAsync(c.wv.p, 0, N * sizeof(double), c.stream));
            k_segaxpy<<<g1, 256, 0, c.stream>>>(kmax, N, C, c.V.p, N, G.y.p, c.vcid.p, 1.0, c.wv.p);
            BEM_LAUNCH_CHECK();
        } else {
            BEM_CUDA(cudaMemsetAsync(c.zv.p, 0, N * sizeof(double), c.stream));
            k_segaxpy<<<g1, 256, 0, c.stream>>>(kmax, N, C, c.V.p, N, G.y.p, c.vcid.p, 1.0, c.zv.p);
            BEM_LAUNCH_CHECK();
            precond_apply(c.zv.p, c.wv.p);
        }
        k_axpby_b<<<g1, 256, 0, c.stream>>>(N, 1.0, c.wv.p, 1.0, x);
        k_axpby_b<<<g1, 256, 0, c.stream>>>(N, 1.0, c.wv.p, 1.0, c.dv.p);
        BEM_LAUNCH_CHECK();
    };

    // per-cluster right-hand-side norms
    segdots(1, b, N, b, G.nrm2.p, 0);
    std::vector<double> bn = read_C(G.nrm2.p);
    for (auto &v : bn) v = std::sqrt(v);
    std::vector<int32_t> done(C, 0), it_c(C, 0), kk(C, 0), act(C, 0);
    std::vector<double> rel(C, 0.0);
    std::vector<int> done_event(C, -1);
    c.res_hist.clear();
    c.cl_events_used = 0;
    auto mark = [&]() {  // an event after the work so far; returns its index
        if (c.cl_events_used == (int)c.cl_events.size()) {
            cudaEvent_t e;
            BEM_CUDA(cudaEventCreate(&e));
            c.cl_events.push_back(e);
        }
        BEM_CUDA(cudaEventRecord(c.cl_events[c.cl_events_used], c.stream));
        return c.cl_events_used++;
    };
    const int ev_start = mark();
    int iters = 0, mvps = 0;
    for (int k = 0; k < C; ++k)
        if (bn[k] == 0.0) {  // zero right-hand side: zero solution
            done[k] = 1;
            rel[k] = 0.0;
        }
    bool zero_any = false;
    for (int k = 0; k < C; ++k) zero_any = zero_any || bn[k] == 0.0;
    if (zero_any) {  // x = 0 on those clusters
        std::vector<int32_t> z(C);
        for (int k = 0; k < C; ++k) z[k] = bn[k] == 0.0;
        upload(G.sel, z);
        k_zero_clusters<<<g1, 256, 0, c.stream>>>(N, c.vcid.p, G.sel.p, x);
        BEM_LAUNCH_CHECK();
    }
    bool have_r = false;
    c.dv.resize(N);
    while (true) {
        // residuals per cluster: r = b - A x on entry, then r = r_0 - A d after each cycle (d the
        // cycle's updates; zero, with a zero product, on clusters it did not update), for the
        // reason given in gmres.cu
        if (!have_r) {
            apply_full(c, 1.0, x, 0.0, nullptr, c.rv.p);
            k_axpby_b<<<g1, 256, 0, c.stream>>>(N, 1.0, b, -1.0, c.rv.p);
        } else {
            apply_full(c, 1.0, c.dv.p, 0.0, nullptr, c.wv.p);
            k_axpby_b<<<g1, 256, 0, c.stream>>>(N, -1.0, c.wv.p, 1.0, c.rv.p);
        }
        ++mvps;
        BEM_LAUNCH_CHECK();
        have_r = true;
        segdots(1, c.rv.p, N, c.rv.p, G.nrm2.p, 0);
        const std::vector<double> beta2 = read_C(G.nrm2.p);
        double worst = 0.0;
        bool all = true;
        for (int k = 0; k < C; ++k) {
            if (bn[k] == 0.0) continue;
            rel[k] = std::sqrt(beta2[k]) / bn[k];
            done[k] = rel[k] <= tol;
            if (done[k] && done_event[k] < 0) done_event[k] = ev_start;  // met on entry
            all = all && done[k];
            worst = std::max(worst, rel[k]);
        }
        c.res_hist.push_back(worst);
        if (all || iters >= maxit) break;
        for (int k = 0; k < C; ++k) act[k] = !done[k];
        upload(G.active, act);
        // v_0 = r / |r| per active cluster, g = (beta, 0, ...)
        k_segnormalise<<<g1, 256, 0, c.stream>>>(N, c.rv.p, G.nrm2.p, c.vcid.p, G.active.p, c.V.p);
        k_cycle_start_b<<<gc, 128, 0, c.stream>>>(m, C, G.nrm2.p, G.g.p);
        BEM_LAUNCH_CHECK();
        BEM_CUDA(cudaMemsetAsync(c.dv.p, 0, N * sizeof(double), c.stream));
        std::fill(kk.begin(), kk.end(), 0);
        std::vector<int32_t> conv(C, 0);  // converged within this cycle (solution already updated)
        for (int k = 0; k < m; ++k) {
            double *vk = c.V.p + (size_t)k * N;
            if (pmode != 0) {
                precond_apply(vk, c.zv.p);
                apply_full(c, 1.0, c.zv.p, 0.0, nullptr, c.wv.p);
            } else {
                apply_full(c, 1.0, vk, 0.0, nullptr, c.wv.p);
            }
            ++mvps;
            // classical Gram-Schmidt twice, per cluster
            segdots(k + 1, c.V.p, N, c.wv.p, G.h.p, 0);
            k_segaxpy<<<g1, 256, 0, c.stream>>>(k + 1, N, C, c.V.p, N, G.h.p, c.vcid.p, -1.0, c.wv.p);
            BEM_LAUNCH_CHECK();
            segdots(k + 1, c.V.p, N, c.wv.p, G.h2.p, 0);
            k_segaxpy<<<g1, 256, 0, c.stream>>>(k + 1, N, C, c.V.p, N, G.h2.p, c.vcid.p, -1.0, c.wv.p);
            k_axpby_b<<<1, 256, 0, c.stream>>>((int64_t)(k + 1) * C, 1.0, G.h2.p, 1.0, G.h.p);
            BEM_LAUNCH_CHECK();
            segdots(1, c.wv.p, N, c.wv.p, G.nrm2.p, 0);
            k_segnormalise<<<g1, 256, 0, c.stream>>>(N, c.wv.p, G.nrm2.p, c.vcid.p, G.active.p,
                                                      c.V.p + (size_t)(k + 1) * N);
            k_givens_b<<<gc, 128, 0, c.stream>>>(k, m, C, G.h.p, G.nrm2.p, G.active.p, G.H.p, G.cs.p, G.sn.p, G.g.p,
                                                 G.res.p);
            BEM_LAUNCH_CHECK();
            ++iters;
            const std::vector<double> est = read_C(G.res.p);
            std::vector<int32_t> now(C, 0);
            bool any_now = false, any_active = false;
            double west = 0.0;
            for (int q = 0; q < C; ++q) {
                if (!act[q]) continue;
                kk[q] = k + 1;
                it_c[q] += 1;
                const double e = est[q] / bn[q];
                west = std::max(west, e);
                if (e <= tol) {
                    now[q] = 1;
                    any_now = true;
                    act[q] = 0;
                    conv[q] = 1;
                } else {
                    any_active = true;
                }
            }
            c.res_hist.push_back(west);
            if (any_now) {
                // the clusters that met the tolerance take their solution now and stop
                update(kk, now);
                const int e = mark();
                for (int q = 0; q < C; ++q)
                    if (now[q]) done_event[q] = e;
                upload(G.active, act);
            }
            if (!any_active || iters >= maxit) break;
        }
        // the clusters still running take the solution of this cycle
        std::vector<int32_t> rest(C, 0);
        bool any_rest = false;
        for (int q = 0; q < C; ++q) {
            rest[q] = act[q] && !conv[q];
            any_rest = any_rest || rest[q];
        }
        if (any_rest) update(kk, rest);
        const int e = mark();
        for (int q = 0; q < C; ++q)
            if (rest[q]) done_event[q] = e;
    }
    BEM_CUDA(cudaStreamSynchronize(c.stream));
    // per-cluster results: iterations, true relative residual, device ms until final
    c.cl_iters.assign(it_c.begin(), it_c.end());
    c.cl_relres = rel;
    c.cl_done_ms.assign(C, 0.0);
    {
        float ms = 0.f;
        BEM_CUDA(cudaEventElapsedTime(&ms, c.cl_events[ev_start], c.cl_events[c.cl_events_used - 1]));
        c.cl_solve_ms = ms;
    }
    for (int q = 0; q < C; ++q) {
        float ms = 0.f;
        if (done_event[q] >= 0) BEM_CUDA(cudaEventElapsedTime(&ms, c.cl_events[ev_start], c.cl_events[done_event[q]]));
        c.cl_done_ms[q] = ms;
    }
    double worst = 0.0;
    bool conv_all = true;
    for (int q = 0; q < C; ++q) {
        worst = std::max(worst, rel[q]);
        conv_all = conv_all && (bn[q] == 0.0 || rel[q] <= tol);
    }
    if (pmode == 2) block_precond_check(c);
    c.stats.last_iters = iters;
    c.stats.last_mvps = mvps;
    c.stats.last_relres = worst;
    if (iters_out) *iters_out = iters;
    if (relres_out) *relres_out = worst;
    if (!conv_all) fail(BEM_ERR_NOCONV, "GMRES reached maxit before every cluster met the tolerance");
}

}  // namespace bem
