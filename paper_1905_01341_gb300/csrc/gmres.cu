// GMRES (Saad and Schultz) for L q = b, Section 3.8, kept on the device in FP64: unpreconditioned
// as in the paper, or right-preconditioned (Jacobi, or the bubble blocks of precond.cu). The Krylov basis V, the Hessenberg matrix, the Givens rotations and the rotated
// right-hand side live in device memory; the host only reads the residual estimate once
// per iteration to decide whether to stop.
//
// Arnoldi uses classical Gram-Schmidt applied twice (one fused multi-dot and one fused
// multi-axpy per pass): the same basis as modified Gram-Schmidt up to rounding, with two
// reads of V per pass instead of one dependent pass per basis vector. All reductions are
// two-stage with a fixed summation order, so a solve is reproducible run to run.
//
// Mixed precision stores the basis in FP32 (a compressed-basis GMRES, after Aliaga, Anzt et
// al.): the work vector, the Hessenberg matrix, the rotations and the iterate stay FP64, each
// v_{k+1} is rounded to FP32 once when it is normalised, and every later use (the product
// A P v_k, the projections, the solution update) reads that same stored vector, so the Arnoldi
// relation holds with the stored basis up to the one rounding of each new vector (~6e-8 of its
// norm, far below the 1e-6 tolerance). The projections V^T w and updates w - V h run in
// compensated FP32 (an exact product of the FP32 basis value with the (hi, lo) split of the
// FP64 operand plus the cross term, summed with TwoSum; about 1e-14 relative), half the bytes
// and none of the FP64 arithmetic of the FP64 basis.
//
// A solve stops on the residual r = b - L q evaluated with operator products, not on GMRES's
// own estimate: the first cycle starts from r_0 = b - A x_0 (a product of the initial iterate),
// and every cycle ends with r = r_0 - A d, d = P V y its update, one product of d. Evaluating
// A on the whole new iterate instead would round x_0 + d to the mixed product's FP32 inputs a
// second time, which moves A x by about 1e-7 of |b| (a tenth of a 1e-6 tolerance) in a direction
// unrelated to the Krylov space, so that a cycle whose estimate met the tolerance could fail the
// check and restart for no gain; r_0 - A d agrees with the estimate to the rounding of A d, and
// the next cycle starts from it.
#include "internal.h"

#include <algorithm>
#include <cmath>

namespace bem {
namespace {

constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 152 * 3;  // fixed grid: fixed summation order
constexpr int RED_JB = 8;            // basis vectors per pass over w

// partial[j * RED_BLOCKS + block] = sum over the block's slice of V_j . w, j = 0..nv-1.
// Each pass reads w once for RED_JB vectors (independent accumulators), then reduces the
// RED_JB sums across the block in a fixed order.
__global__ void __launch_bounds__(RED_THREADS) k_multidot(int nv, int64_t N, const double *__restrict__ V,
                                                          size_t ldv, const double *__restrict__ w,
                                                          double *__restrict__ partial) {
    __shared__ double red[RED_THREADS / 32][RED_JB];
    const int64_t chunk = (N + RED_BLOCKS - 1) / RED_BLOCKS;
    const int64_t i0 = blockIdx.x * chunk, i1 = (N < i0 + chunk) ? N : i0 + chunk;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j0 = 0; j0 < nv; j0 += RED_JB) {
        const int nj = min(RED_JB, nv - j0);
        double s[RED_JB];
#pragma unroll
        for (int jj = 0; jj < RED_JB; ++jj) s[jj] = 0.0;
#pragma unroll 4
        for (int64_t i = i0 + threadIdx.x; i < i1; i += RED_THREADS) {
            const double wi = w[i];
#pragma unroll
            for (int jj = 0; jj < RED_JB; ++jj)
                if (jj < nj) s[jj] = fma(V[(size_t)(j0 + jj) * ldv + i], wi, s[jj]);
        }
#pragma unroll
        for (int jj = 0; jj < RED_JB; ++jj) {
            double t = s[jj];
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) red[warp][jj] = t;
        }
        __syncthreads();
        if (threadIdx.x < nj) {
            double t = 0.0;
            for (int k = 0; k < RED_THREADS / 32; ++k) t += red[k][threadIdx.x];
            partial[(size_t)(j0 + threadIdx.x) * RED_BLOCKS + blockIdx.x] = t;
        }
        __syncthreads();
    }
}

// out[j] = (accumulate ? out[j] : 0) + sum_b partial[j][b]  (one block per j; fixed order)
__global__ void k_dot_final(const double *__restrict__ partial, double *__restrict__ out, int accumulate) {
    __shared__ double red[RED_THREADS];
    double s = 0.0;
    for (int b = threadIdx.x; b < RED_BLOCKS; b += RED_THREADS) s += partial[(size_t)blockIdx.x * RED_BLOCKS + b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = RED_THREADS / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = (accumulate ? out[blockIdx.x] : 0.0) + red[0];
}

// w -= sum_j h[j] V_j  (sign = -1) or w += ... (sign = +1)
__global__ void k_multiaxpy(int nv, int64_t N, const double *__restrict__ V, size_t ldv,
                            const double *__restrict__ h, double sign, double *__restrict__ w) {
    __shared__ double hs[128];
    if (threadIdx.x < nv) hs[threadIdx.x] = h[threadIdx.x];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
#pragma unroll 8
        for (int j = 0; j < nv; ++j) acc = fma(hs[j], V[j * ldv + i], acc);
        w[i] += sign * acc;
    }
}

// s + c += p + e with TwoSum (e: the product's rounding error, added to the compensation)
__device__ __forceinline__ void two_sum_acc(float &s, float &c, float p, float e) {
    const float t = s + p, bp = t - s;
    c += ((s - (t - bp)) + (p - bp)) + e;
    s = t;
}

// k_multidot with an FP32 basis: partial[j * RED_BLOCKS + block] = the block's share of V_j . w,
// compensated FP32 per thread, the (sum, compensation) pairs joined in a fixed order
__global__ void __launch_bounds__(RED_THREADS) k_multidot32(int nv, int64_t N, const float *__restrict__ V,
                                                            size_t ldv, const double *__restrict__ w,
                                                            double *__restrict__ partial) {
    __shared__ float red[2][RED_THREADS / 32][RED_JB];
    const int64_t chunk = (N + RED_BLOCKS - 1) / RED_BLOCKS;
    const int64_t i0 = blockIdx.x * chunk, i1 = (N < i0 + chunk) ? N : i0 + chunk;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j0 = 0; j0 < nv; j0 += RED_JB) {
        const int nj = min(RED_JB, nv - j0);
        float s[RED_JB], c[RED_JB];
#pragma unroll
        for (int jj = 0; jj < RED_JB; ++jj) s[jj] = c[jj] = 0.f;
#pragma unroll 4
        for (int64_t i = i0 + threadIdx.x; i < i1; i += RED_THREADS) {
            const double wi = w[i];
            const float wh = (float)wi, wl = (float)(wi - (double)wh);
#pragma unroll
            for (int jj = 0; jj < RED_JB; ++jj)
                if (jj < nj) {
                    const float v = V[(size_t)(j0 + jj) * ldv + i];
                    const float p = v * wh;
                    two_sum_acc(s[jj], c[jj], p, fmaf(v, wl, fmaf(v, wh, -p)));
                }
        }
#pragma unroll
        for (int jj = 0; jj < RED_JB; ++jj) {
            float t = s[jj], u = c[jj];
            for (int o = 16; o > 0; o >>= 1) {
                const float ot = __shfl_down_sync(0xffffffffu, t, o), ou = __shfl_down_sync(0xffffffffu, u, o);
                two_sum_acc(t, u, ot, ou);
            }
            if (lane == 0) {
                red[0][warp][jj] = t;
                red[1][warp][jj] = u;
            }
        }
        __syncthreads();
        if (threadIdx.x < nj) {
            double t = 0.0;
            for (int k = 0; k < RED_THREADS / 32; ++k) t += (double)red[0][k][threadIdx.x] + (double)red[1][k][threadIdx.x];
            partial[(size_t)(j0 + threadIdx.x) * RED_BLOCKS + blockIdx.x] = t;
        }
        __syncthreads();
    }
}

// k_multiaxpy with an FP32 basis: w += sign * sum_j h[j] V_j, the sum in compensated FP32 with
// h split into (hi, lo) pairs, added to the FP64 w once per element
__global__ void k_multiaxpy32(int nv, int64_t N, const float *__restrict__ V, size_t ldv,
                              const double *__restrict__ h, double sign, double *__restrict__ w) {
    __shared__ float2 hs[128];
    if (threadIdx.x < nv) {
        const double hv = h[threadIdx.x];
        const float hh = (float)hv;
        hs[threadIdx.x] = make_float2(hh, (float)(hv - (double)hh));
    }
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f, c = 0.f;
#pragma unroll 8
        for (int j = 0; j < nv; ++j) {
            const float v = V[(size_t)j * ldv + i];
            const float2 g = hs[j];
            const float p = g.x * v;
            two_sum_acc(s, c, p, fmaf(g.y, v, fmaf(g.x, v, -p)));
        }
        w[i] += sign * ((double)s + (double)c);
    }
}

// v = (float)(w / sqrt(nrm2[0])) into the FP32 basis, and its exact FP64 copy for the product
__global__ void k_normalise32(int64_t N, const double *__restrict__ w, const double *__restrict__ nrm2,
                              float *__restrict__ v, double *__restrict__ v64, double *__restrict__ out_norm) {
    double nn = sqrt(fmax(nrm2[0], 0.0));
    double inv = nn > 0.0 ? 1.0 / nn : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const float f = (float)(w[i] * inv);
        v[i] = f;
        v64[i] = (double)f;
    }
    if (out_norm && blockIdx.x == 0 && threadIdx.x == 0) *out_norm = nn;
}

// y = alpha * x + beta * y
__global__ void k_axpby(int64_t N, double alpha, const double *__restrict__ x, double beta, double *__restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = alpha * x[i] + beta * y[i];
}

// v = w / sqrt(nrm2[0]); writes the norm to out_norm (when set). Zero norm gives v = 0.
__global__ void k_normalise(int64_t N, const double *__restrict__ w, const double *__restrict__ nrm2,
                            double *__restrict__ v, double *__restrict__ out_norm) {
    double nn = sqrt(fmax(nrm2[0], 0.0));
    double inv = nn > 0.0 ? 1.0 / nn : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = w[i] * inv;
    if (out_norm && blockIdx.x == 0 && threadIdx.x == 0) *out_norm = nn;
}

// Start of a cycle: g = (beta, 0, ...), rotations cleared. scal[0] = beta.
__global__ void k_cycle_start(int m, const double *__restrict__ beta, double *__restrict__ g) {
    for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = (i == 0) ? beta[0] : 0.0;
}

// Column k of the Hessenberg matrix (h[0..k] from Gram-Schmidt, hk1 = h[k+1]) through the
// previous rotations, a new rotation that zeroes h[k+1], and the rotated right-hand side.
// H is stored column-major with leading dimension m+1. resid[0] = |g[k+1]|.
__global__ void k_givens(int k, int m, const double *__restrict__ h, double *__restrict__ H,
                         double *__restrict__ cs, double *__restrict__ sn, double *__restrict__ g,
                         double *__restrict__ resid) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double *col = H + (size_t)k * (m + 1);
    for (int i = 0; i <= k + 1; ++i) col[i] = h[i];
    for (int j = 0; j < k; ++j) {
        double t = cs[j] * col[j] + sn[j] * col[j + 1];
        col[j + 1] = -sn[j] * col[j] + cs[j] * col[j + 1];
        col[j] = t;
    }
    double d = hypot(col[k], col[k + 1]);
    double c = 1.0, s = 0.0;
    if (d != 0.0) {
        c = col[k] / d;
        s = col[k + 1] / d;
    }
    cs[k] = c;
    sn[k] = s;
    col[k] = d;
    col[k + 1] = 0.0;
    g[k + 1] = -s * g[k];
    g[k] = c * g[k];
    resid[0] = fabs(g[k + 1]);
}

// z = d .* v (right preconditioning by the inverse diagonal)
__global__ void k_scale_by(int64_t N, const double *__restrict__ d, const double *__restrict__ v, double *__restrict__ z) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        z[i] = v[i] / d[i];
}


// Back substitution: H(0:kk,0:kk) y = g(0:kk).
__global__ void k_backsolve(int kk, int m, const double *__restrict__ H, const double *__restrict__ g,
                            double *__restrict__ y) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = kk - 1; i >= 0; --i) {
        double s = g[i];
        for (int j = i + 1; j < kk; ++j) s -= H[(size_t)j * (m + 1) + i] * y[j];
        double d = H[(size_t)i * (m + 1) + i];
        y[i] = d != 0.0 ? s / d : 0.0;
    }
}

struct Vec {
    Context &c;
    int64_t N;
    int grid;
    explicit Vec(Context &cc) : c(cc), N(cc.N) { grid = std::min<int64_t>(div_up(N, 256), 152 * 8); }
    // out[0..nv) = V_j . w (deterministic)
    void dots(int nv, const double *V, size_t ldv, const double *w, double *out, int accumulate) {
        PhaseScope ps(c, PH_GMRES);
        k_multidot<<<RED_BLOCKS, RED_THREADS, 0, c.stream>>>(nv, N, V, ldv, w, c.partial.p);
        BEM_LAUNCH_CHECK();
        k_dot_final<<<nv, RED_THREADS, 0, c.stream>>>(c.partial.p, out, accumulate);
        BEM_LAUNCH_CHECK();
    }
    void multiaxpy(int nv, const double *V, size_t ldv, const double *h, double sign, double *w) {
        PhaseScope ps(c, PH_GMRES);
        k_multiaxpy<<<grid, 256, 0, c.stream>>>(nv, N, V, ldv, h, sign, w);
        BEM_LAUNCH_CHECK();
    }
    // the same with the FP32 basis
    void dots(int nv, const float *V, size_t ldv, const double *w, double *out, int accumulate) {
        PhaseScope ps(c, PH_GMRES);
        k_multidot32<<<RED_BLOCKS, RED_THREADS, 0, c.stream>>>(nv, N, V, ldv, w, c.partial.p);
        BEM_LAUNCH_CHECK();
        k_dot_final<<<nv, RED_THREADS, 0, c.stream>>>(c.partial.p, out, accumulate);
        BEM_LAUNCH_CHECK();
    }
    void multiaxpy(int nv, const float *V, size_t ldv, const double *h, double sign, double *w) {
        PhaseScope ps(c, PH_GMRES);
        k_multiaxpy32<<<grid, 256, 0, c.stream>>>(nv, N, V, ldv, h, sign, w);
        BEM_LAUNCH_CHECK();
    }
    // v_k = w / |w| into the basis (FP64, or FP32 with the FP64 copy v64); |w| to out_norm
    void normalise(const double *w, const double *nrm2, double *V, float *V32, int k, double *v64,
                   double *out_norm) {
        PhaseScope ps(c, PH_GMRES);
        if (V32)
            k_normalise32<<<grid, 256, 0, c.stream>>>(N, w, nrm2, V32 + (size_t)k * N, v64, out_norm);
        else
            k_normalise<<<grid, 256, 0, c.stream>>>(N, w, nrm2, V + (size_t)k * N, out_norm);
        BEM_LAUNCH_CHECK();
    }
    void axpby(double a, const double *x, double b, double *y) {
        PhaseScope ps(c, PH_GMRES);
        k_axpby<<<grid, 256, 0, c.stream>>>(N, a, x, b, y);
        BEM_LAUNCH_CHECK();
    }
};

double read_scalar(Context &c, const double *dev) {
    double *h = c.hscal.get(1);
    BEM_CUDA(cudaMemcpyAsync(h, dev, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    BEM_CUDA(cudaStreamSynchronize(c.stream));
    return *h;
}

}  // namespace

// x holds the initial guess on entry and the solution on exit (device, caller order).
void gmres_solve(Context &c, const double *b, double *x, int *iters_out, double *relres_out) {
    const int64_t N = c.N;
    const int maxit = std::max(1, c.prm.gmres_maxit);
    // restart length: the caller's, else no restart up to 127 basis vectors
    const int m = std::min({maxit, c.prm.gmres_restart > 0 ? c.prm.gmres_restart : maxit, 127});
    const double tol = c.prm.gmres_tol;
    Vec vec(c);
    const int pmode = c.prm.gmres_precond;  // 0 none, 1 Jacobi, 2 bubble blocks
    const bool precond = pmode != 0;
    if (precond) c.zv.resize(N);
    if (pmode == 2) block_precond_prepare(c);
    const bool b32 = c.prm.precision != BEM_PREC_FP64;  // the basis in FP32 (mixed precision)
    if (b32) {
        c.V32.resize((size_t)(m + 1) * N);
        c.vk64.resize(N);
    } else {
        c.V.resize((size_t)(m + 1) * N);
    }
    auto project = [&](int nv, const double *w, double *out) {
        if (b32) vec.dots(nv, (const float *)c.V32.p, N, w, out, 0);
        else vec.dots(nv, (const double *)c.V.p, N, w, out, 0);
    };
    auto update = [&](int nv, const double *h, double sign, double *w) {
        if (b32) vec.multiaxpy(nv, (const float *)c.V32.p, N, h, sign, w);
        else vec.multiaxpy(nv, (const double *)c.V.p, N, h, sign, w);
    };
    c.wv.resize(N);
    c.rv.resize(N);
    c.partial.resize((size_t)(m + 2) * RED_BLOCKS);
    c.hcol.resize(m + 2);
    c.hmat.resize((size_t)(m + 1) * (m + 1));
    c.givens.resize(2 * (m + 1));
    c.gvec.resize(m + 2);
    c.yvec.resize(m + 1);
    c.scal.resize(8);
    double *cs = c.givens.p, *sn = c.givens.p + (m + 1);
    double *d_bn2 = c.scal.p, *d_beta2 = c.scal.p + 1, *d_beta = c.scal.p + 2, *d_res = c.scal.p + 3;
    double *d_tmp = c.scal.p + 4;

    c.res_hist.clear();
    vec.dots(1, b, N, b, d_bn2, 0);
    const double bnorm = std::sqrt(read_scalar(c, d_bn2));
    int iters = 0, mvps = 0;
    double relres = 0.0;
    if (bnorm == 0.0) {
        BEM_CUDA(cudaMemsetAsync(x, 0, N * sizeof(double), c.stream));
        c.stats.last_iters = 0;
        c.stats.last_mvps = 0;
        c.stats.last_relres = 0.0;
        if (iters_out) *iters_out = 0;
        if (relres_out) *relres_out = 0.0;
        return;
    }
    bool converged = false, have_r = false;
    c.dv.resize(N);
    while (true) {
        if (!have_r) {  // r = b - A x, the product of the full iterate (the first cycle's start)
            apply_full(c, 1.0, x, 0.0, nullptr, c.rv.p);
            ++mvps;
            vec.axpby(1.0, b, -1.0, c.rv.p);
        }
        vec.dots(1, c.rv.p, N, c.rv.p, d_beta2, 0);
        double beta = std::sqrt(read_scalar(c, d_beta2));
        relres = beta / bnorm;
        c.res_hist.push_back(relres);
        if (relres <= tol) {
            converged = true;
            break;
        }
        if (iters >= maxit) break;
        vec.normalise(c.rv.p, d_beta2, c.V.p, b32 ? c.V32.p : nullptr, 0, c.vk64.p, d_beta);
        k_cycle_start<<<1, 128, 0, c.stream>>>(m, d_beta, c.gvec.p);
        BEM_LAUNCH_CHECK();
        int kk = 0;
        for (int k = 0; k < m; ++k) {
            const double *vk = b32 ? c.vk64.p : c.V.p + (size_t)k * N;  // the stored v_k
            if (pmode == 1) {  // w = A D^-1 v_k
                k_scale_by<<<vec.grid, 256, 0, c.stream>>>(N, c.ldiag.p, vk, c.zv.p);
                BEM_LAUNCH_CHECK();
                apply_full(c, 1.0, c.zv.p, 0.0, nullptr, c.wv.p);
            } else if (pmode == 2) {  // w = A P v_k
                {
                    PhaseScope ps(c, PH_GMRES);
                    block_precond_apply(c, vk, c.zv.p);
                }
                apply_full(c, 1.0, c.zv.p, 0.0, nullptr, c.wv.p);
            } else {
                apply_full(c, 1.0, vk, 0.0, nullptr, c.wv.p);
            }
            ++mvps;
            // classical Gram-Schmidt, twice
            project(k + 1, c.wv.p, c.hcol.p);
            update(k + 1, c.hcol.p, -1.0, c.wv.p);
            project(k + 1, c.wv.p, c.yvec.p);  // second pass into y (free here)
            update(k + 1, c.yvec.p, -1.0, c.wv.p);
            k_axpby<<<1, 128, 0, c.stream>>>(k + 1, 1.0, c.yvec.p, 1.0, c.hcol.p);
            BEM_LAUNCH_CHECK();
            vec.dots(1, c.wv.p, N, c.wv.p, d_tmp, 0);
            // h[k+1] = |w|, v_{k+1} = w / |w|
            vec.normalise(c.wv.p, d_tmp, c.V.p, b32 ? c.V32.p : nullptr, k + 1, c.vk64.p, c.hcol.p + k + 1);
            k_givens<<<1, 1, 0, c.stream>>>(k, m, c.hcol.p, c.hmat.p, cs, sn, c.gvec.p, d_res);
            BEM_LAUNCH_CHECK();
            ++iters;
            kk = k + 1;
            double est = read_scalar(c, d_res) / bnorm;
            c.res_hist.push_back(est);
            if (est <= tol || iters >= maxit) break;
        }
        k_backsolve<<<1, 1, 0, c.stream>>>(kk, m, c.hmat.p, c.gvec.p, c.yvec.p);
        BEM_LAUNCH_CHECK();
        // the cycle's update d = P V y (P = D^-1, the bubble blocks or the identity), x += d
        if (pmode == 1) {
            BEM_CUDA(cudaMemsetAsync(c.zv.p, 0, N * sizeof(double), c.stream));
            update(kk, c.yvec.p, 1.0, c.zv.p);
            k_scale_by<<<vec.grid, 256, 0, c.stream>>>(N, c.ldiag.p, c.zv.p, c.dv.p);
            BEM_LAUNCH_CHECK();
        } else if (pmode == 2) {
            BEM_CUDA(cudaMemsetAsync(c.zv.p, 0, N * sizeof(double), c.stream));
            update(kk, c.yvec.p, 1.0, c.zv.p);
            PhaseScope ps(c, PH_GMRES);
            block_precond_apply(c, c.zv.p, c.dv.p);
        } else {
            BEM_CUDA(cudaMemsetAsync(c.dv.p, 0, N * sizeof(double), c.stream));
            update(kk, c.yvec.p, 1.0, c.dv.p);
        }
        vec.axpby(1.0, c.dv.p, 1.0, x);
        // r = r_0 - A d: the product of the update, not of the whole iterate (see the header)
        apply_full(c, 1.0, c.dv.p, 0.0, nullptr, c.wv.p);
        ++mvps;
        vec.axpby(-1.0, c.wv.p, 1.0, c.rv.p);
        have_r = true;
    }
    if (pmode == 2) block_precond_check(c);
    c.stats.last_iters = iters;
    c.stats.last_mvps = mvps;
    c.stats.last_relres = relres;
    if (iters_out) *iters_out = iters;
    if (relres_out) *relres_out = relres;
    if (!converged) fail(BEM_ERR_NOCONV, "GMRES reached maxit without meeting the tolerance");
}

}  // namespace bem
