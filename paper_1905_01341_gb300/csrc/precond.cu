// Bubble-block preconditioner for the GMRES solve of L q = b (gmres_precond = 2).
//
// The paper solves with unpreconditioned GMRES and mentions a preconditioned flexible GMRES
// as the alternative it tried (Section 3.8). The slow GMRES components here are those of each
// bubble's own single-layer block: on a sphere of radius R its eigenvalues are R/(2n+1), a
// spread that grows with the mesh resolution. This preconditioner removes them: for every
// distinct bubble mesh (same connectivity; every icosphere of one level is one group), it
// inverts the single-layer matrix of the isolated representative bubble, including its
// singular diagonal from the identity of Eq. (s5) summed over that bubble alone, and scales
// it to unit size. Bubble m of the group is
// preconditioned by (1/R_m) times that inverse, R_m its current mean centroid distance (the
// single layer of a bubble scaled by R is R times the unit one). The inverse is built from
// the geometry of the first solve after a mesh upload and kept; only the scales follow the
// bubbles as they move. The solve still stops on the true residual |b - L q| / |b| of the
// unpreconditioned system, so the solution meets the same tolerance.
//
// Setup per shape (n vertices): the n x n block is assembled in FP64 and inverted in place by
// Gauss-Jordan elimination without pivoting (two launches per pivot). The block is K S with K
// the symmetric single-layer kernel matrix and S the diagonal of vertex areas, so every
// leading principal minor is positive when K is positive definite; a pivot that is not
// positive stops the setup with an error. Apply: one tiled GEMM per shape, FP32 on the mixed
// path and FP64 on the FP64 path, with the bubbles' vertex ranges as the right-hand columns.
#include "internal.h"

#include <cmath>

namespace bem {
namespace {

constexpr double kInv4Pi = 0.0795774715459476678844418816862571810;

// Row i of the isolated bubble's single-layer block (vertices a..a+n-1 in caller order),
// coordinates relative to the centroid c: A_ij = s_j / (4 pi |r_i - r_j|) for j != i and
// A_ii = n_i . [ sum_{j != i} (M_ij r_j - L_ij n_j) + (1/2 + M_ii) r_i ], M_ii = -1/2 - sum M_ij,
// all sums over this bubble only (Eqs. (s3), (s5)).
__global__ void k_bp_assemble(int n, int64_t N, int64_t a, double cx, double cy, double cz,
                              const double *__restrict__ xyz, const double *__restrict__ s,
                              const double *__restrict__ nrm, double *__restrict__ A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t gi = a + i;
    const double xi = xyz[gi] - cx, yi = xyz[N + gi] - cy, zi = xyz[2 * N + gi] - cz;
    double msum = 0.0, vx = 0.0, vy = 0.0, vz = 0.0;
    for (int j = 0; j < n; ++j) {
        if (j == i) continue;
        const int64_t gj = a + j;
        const double xj = xyz[gj] - cx, yj = xyz[N + gj] - cy, zj = xyz[2 * N + gj] - cz;
        const double dx = xi - xj, dy = yi - yj, dz = zi - zj;
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double rinv = 1.0 / sqrt(r2);
        const double nx = nrm[gj], ny = nrm[N + gj], nz = nrm[2 * N + gj];
        const double lij = s[gj] * kInv4Pi * rinv;
        const double mij = s[gj] * kInv4Pi * (nx * dx + ny * dy + nz * dz) * rinv * rinv * rinv;
        A[(size_t)i * n + j] = lij;
        msum += mij;
        vx += mij * xj - lij * nx;
        vy += mij * yj - lij * ny;
        vz += mij * zj - lij * nz;
    }
    const double mii = -0.5 - msum;
    const double h = 0.5 + mii;
    A[(size_t)i * n + i] = nrm[gi] * (vx + h * xi) + nrm[N + gi] * (vy + h * yi) + nrm[2 * N + gi] * (vz + h * zi);
}

// Gauss-Jordan step k, part 1: A_ij -= A_ik A_kj / A_kk for i != k and j != k (row k and column
// k are read, not written); keeps a copy of the pivot for part 2.
__global__ void k_gj_interior(int n, int k, double *__restrict__ A, double *__restrict__ piv) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    const double p = A[(size_t)k * n + k];
    if (i == 0 && j == 0) *piv = p;
    if (i == k || j >= n || j == k) return;
    A[(size_t)i * n + j] -= A[(size_t)i * n + k] * A[(size_t)k * n + j] / p;
}

// Gauss-Jordan step k, part 2: row k /= p, column k = -column k / p, A_kk = 1 / p.
__global__ void k_gj_pivot(int n, int k, double *__restrict__ A, const double *__restrict__ piv,
                           int *__restrict__ bad) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const double p = *piv;
    if (t == 0 && !(p > 0.0)) atomicOr(bad, 1);
    if (t >= n) return;
    if (t == k) {
        A[(size_t)k * n + k] = 1.0 / p;
    } else {
        A[(size_t)k * n + t] /= p;
        A[(size_t)t * n + k] = -A[(size_t)t * n + k] / p;
    }
}

// inverse at size R -> unit size (times R), FP64 and FP32 copies
__global__ void k_bp_store(size_t cnt, double R, const double *__restrict__ A, double *__restrict__ o64,
                           float *__restrict__ o32) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < cnt; e += (size_t)gridDim.x * blockDim.x) {
        const double v = A[e] * R;
        o64[e] = v;
        o32[e] = (float)v;
    }
}

// per bubble of a shape (one block each): 1 / mean distance of its vertices from their centroid
__global__ void k_bp_scales(int n, int64_t N, const int64_t *__restrict__ voff, const double *__restrict__ xyz,
                            double *__restrict__ scale) {
    __shared__ double red[4][8];
    const int64_t a = voff[blockIdx.x];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        sx += xyz[a + i];
        sy += xyz[N + a + i];
        sz += xyz[2 * N + a + i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_down_sync(0xffffffffu, sx, o);
        sy += __shfl_down_sync(0xffffffffu, sy, o);
        sz += __shfl_down_sync(0xffffffffu, sz, o);
    }
    if (lane == 0) {
        red[0][w] = sx;
        red[1][w] = sy;
        red[2][w] = sz;
    }
    __syncthreads();
    double cx = 0.0, cy = 0.0, cz = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
        cx += red[0][k];
        cy += red[1][k];
        cz += red[2][k];
    }
    cx /= n;
    cy /= n;
    cz /= n;
    double d = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double dx = xyz[a + i] - cx, dy = xyz[N + a + i] - cy, dz = xyz[2 * N + a + i] - cz;
        d += sqrt(dx * dx + dy * dy + dz * dz);
    }
    for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
    __syncthreads();
    if (lane == 0) red[3][w] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[3][k];
        scale[blockIdx.x] = (double)n / t;
    }
}

// z[voff_b + r] = scale_b * sum_k inv[r][k] y[voff_b + k] for the bubbles b of one shape:
// a 64-row x 32-bubble output tile per block, K in steps of 32 through shared memory.
constexpr int BP_TM = 64, BP_TN = 32, BP_TK = 32, BP_THREADS = 256;

template <class T>
__global__ void __launch_bounds__(BP_THREADS) k_bp_apply(int n, const T *__restrict__ inv, int nb,
                                                         const int64_t *__restrict__ voff,
                                                         const double *__restrict__ scale,
                                                         const double *__restrict__ y, double *__restrict__ z) {
    __shared__ T As[BP_TK][BP_TM + 1];
    __shared__ T Bs[BP_TK][BP_TN + 1];
    __shared__ int64_t sv[BP_TN];
    const int row0 = blockIdx.x * BP_TM, b0 = blockIdx.y * BP_TN;
    const int tid = threadIdx.x, tr = tid & 15, tb = tid >> 4;  // rows tr + 16 i, bubbles 2 tb + j
    if (tid < BP_TN) sv[tid] = (b0 + tid < nb) ? voff[b0 + tid] : -1;
    T acc[4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = (T)0;
    for (int k0 = 0; k0 < n; k0 += BP_TK) {
        __syncthreads();
        for (int e = tid; e < BP_TM * BP_TK; e += BP_THREADS) {
            const int r = e / BP_TK, kk = e % BP_TK;
            As[kk][r] = (row0 + r < n && k0 + kk < n) ? inv[(size_t)(row0 + r) * n + k0 + kk] : (T)0;
        }
        for (int e = tid; e < BP_TN * BP_TK; e += BP_THREADS) {
            const int bb = e / BP_TK, kk = e % BP_TK;
            const int64_t v = sv[bb];
            Bs[kk][bb] = (v >= 0 && k0 + kk < n) ? (T)y[v + k0 + kk] : (T)0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < BP_TK; ++kk) {
            const T b0v = Bs[kk][2 * tb], b1v = Bs[kk][2 * tb + 1];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const T av = As[kk][tr + 16 * i];
                acc[i][0] += av * b0v;
                acc[i][1] += av * b1v;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int bb = 2 * tb + j;
        const int64_t v = sv[bb];
        if (v < 0) continue;
        const double sc = scale[b0 + bb];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = row0 + tr + 16 * i;
            if (r < n) z[v + r] = sc * (double)acc[i][j];
        }
    }
}

// FP32 form of the block product: the right-hand side is converted to FP32 once per
// application (k_to_f32), then z_b = s_b Inv y_b for all bubbles of one shape as a tiled GEMM:
// 128 rows x 64 bubbles per block, K in steps of 16 through shared memory, 8 rows x 4 bubbles
// per thread (rows tx*4 + {0..3} and 64 + tx*4 + {0..3}, bubbles ty*4 + {0..3}) read as 16-byte
// vectors, FP32 accumulation in a fixed order.
constexpr int BPF_TM = 128, BPF_TN = 64, BPF_TK = 16, BPF_THREADS = 256;
__global__ void k_to_f32(int64_t n, const double *__restrict__ y, float *__restrict__ yf) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        yf[i] = (float)y[i];
}
__global__ void __launch_bounds__(BPF_THREADS) k_bp_apply_f32(int n, const float *__restrict__ inv, int nb,
                                                              const int64_t *__restrict__ voff,
                                                              const double *__restrict__ scale,
                                                              const float *__restrict__ yf, double *__restrict__ z) {
    // rows padded by 4 floats: the tile loads (consecutive threads along k) hit two banks at most,
    // and rows stay 16-byte aligned for the vector reads
    __shared__ __align__(16) float As[BPF_TK][BPF_TM + 4];
    __shared__ __align__(16) float Bs[BPF_TK][BPF_TN + 4];
    __shared__ int64_t sv[BPF_TN];
    const int row0 = blockIdx.x * BPF_TM, b0 = blockIdx.y * BPF_TN;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    if (tid < BPF_TN) sv[tid] = (b0 + tid < nb) ? voff[b0 + tid] : -1;
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < n; k0 += BPF_TK) {
        __syncthreads();
        for (int e = tid; e < BPF_TM * BPF_TK; e += BPF_THREADS) {  // As[kk][r] = Inv[row0 + r][k0 + kk]
            const int r = e / BPF_TK, kk = e % BPF_TK;
            As[kk][r] = (row0 + r < n && k0 + kk < n) ? inv[(size_t)(row0 + r) * n + k0 + kk] : 0.f;
        }
        for (int e = tid; e < BPF_TN * BPF_TK; e += BPF_THREADS) {  // Bs[kk][b] = y_b[k0 + kk]
            const int bb = e / BPF_TK, kk = e % BPF_TK;
            const int64_t v = sv[bb];
            Bs[kk][bb] = (v >= 0 && k0 + kk < n) ? yf[v + k0 + kk] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BPF_TK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[kk][tx * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[kk][64 + tx * 4]);
            const float4 bv = *reinterpret_cast<const float4 *>(&Bs[kk][ty * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int bb = ty * 4 + j;
        const int64_t v = sv[bb];
        if (v < 0) continue;
        const double sc = scale[b0 + bb];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = row0 + (i < 4 ? tx * 4 + i : 64 + tx * 4 + (i - 4));
            if (r < n) z[v + r] = sc * (double)acc[i][j];
        }
    }
}

// Bubbles whose meshes have the same connectivity (vertex count and triangle list relative to
// their first vertex) share one block inverse: the representative's, scaled by size. A mesh
// copied from one template (every icosphere of one level) is one group however it deforms.
void find_topologies(const Context &c, const std::vector<double> &hx, const std::vector<int32_t> &ht,
                     std::vector<BubbleShape> &shapes, std::vector<int32_t> &shape_of) {
    const int64_t N = c.N, M = c.M, T = c.T;
    shapes.clear();
    shape_of.assign(M, 0);
    for (int64_t m = 0; m < M; ++m) {
        const int64_t a = c.vert_off[m], nd = c.vert_off[m + 1] - a;
        const int64_t ta = c.tri_off[m], nt = c.tri_off[m + 1] - ta;
        int found = -1;
        for (size_t k = 0; k < shapes.size() && found < 0; ++k) {
            const int64_t r = shapes[k].rep;
            const int64_t ra = c.vert_off[r], rta = c.tri_off[r];
            if (shapes[k].nd != nd || c.tri_off[r + 1] - rta != nt) continue;
            bool same = true;
            for (int64_t t = 0; t < nt && same; ++t)
                for (int d = 0; d < 3 && same; ++d) same = ht[d * T + ta + t] - a == ht[d * T + rta + t] - ra;
            if (same) found = (int)k;
        }
        if (found < 0) {
            double cx = 0, cy = 0, cz = 0;
            for (int64_t j = a; j < a + nd; ++j) {
                cx += hx[j];
                cy += hx[N + j];
                cz += hx[2 * N + j];
            }
            shapes.push_back({m, (int)nd, cx / nd, cy / nd, cz / nd});
            found = (int)shapes.size() - 1;
        }
        shape_of[m] = found;
    }
}

void build(Context &c) {
    cudaStream_t st = c.stream;
    const int64_t N = c.N, M = c.M;
    auto &bp = c.bp;
    std::vector<double> hx(3 * N);
    std::vector<int32_t> ht(3 * (size_t)c.T);
    BEM_CUDA(cudaMemcpyAsync(hx.data(), c.xyz.p, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, st));
    BEM_CUDA(cudaMemcpyAsync(ht.data(), c.tri.p, 3 * (size_t)c.T * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    BEM_CUDA(cudaStreamSynchronize(st));
    std::vector<BubbleShape> shapes;
    std::vector<int32_t> shape_of;
    find_topologies(c, hx, ht, shapes, shape_of);
    const size_t ns = shapes.size();
    bp.nd.assign(ns, 0);
    bp.inv_off.assign(ns + 1, 0);
    for (size_t k = 0; k < ns; ++k) {
        bp.nd[k] = shapes[k].nd;
        bp.inv_off[k + 1] = bp.inv_off[k] + (int64_t)shapes[k].nd * shapes[k].nd;
    }
    if (bp.inv_off.back() > (int64_t)1 << 30)
        fail(BEM_ERR_ARG, "bubble-block preconditioner: too many distinct bubble meshes (inverse over 8 GiB)");
    // bubbles grouped by shape
    bp.first.assign(ns + 1, 0);
    for (int64_t m = 0; m < M; ++m) bp.first[shape_of[m] + 1] += 1;
    for (size_t k = 0; k < ns; ++k) bp.first[k + 1] += bp.first[k];
    std::vector<int64_t> grouped(M), fill(bp.first.begin(), bp.first.end() - 1);
    for (int64_t m = 0; m < M; ++m) grouped[fill[shape_of[m]]++] = c.vert_off[m];
    bp.bub_voff.resize(M);
    bp.bub_scale.resize(M);
    BEM_CUDA(cudaMemcpyAsync(bp.bub_voff.p, grouped.data(), M * sizeof(int64_t), cudaMemcpyHostToDevice, st));

    bp.inv64.resize(bp.inv_off.back());
    bp.inv32.resize(bp.inv_off.back());
    int ndmax = 0;
    for (auto &sh : shapes) ndmax = std::max(ndmax, sh.nd);
    DevBuf<double> A, piv;
    DevBuf<int> bad;
    A.resize((size_t)ndmax * ndmax);
    piv.resize(1);
    bad.resize(1);
    BEM_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
    for (size_t k = 0; k < ns; ++k) {
        const BubbleShape &sh = shapes[k];
        const int n = sh.nd;
        const int64_t a = c.vert_off[sh.rep];
        double R = 0.0;  // mean centroid distance of the representative
        for (int i = 0; i < n; ++i) {
            const double dx = hx[a + i] - sh.cx, dy = hx[N + a + i] - sh.cy, dz = hx[2 * N + a + i] - sh.cz;
            R += std::sqrt(dx * dx + dy * dy + dz * dz);
        }
        R /= n;
        k_bp_assemble<<<div_up(n, 128), 128, 0, st>>>(n, N, a, sh.cx, sh.cy, sh.cz, c.xyz.p, c.s.p, c.nrm.p, A.p);
        BEM_LAUNCH_CHECK();
        const dim3 gi((unsigned)div_up(n, 256), (unsigned)n);
        for (int p = 0; p < n; ++p) {
            k_gj_interior<<<gi, 256, 0, st>>>(n, p, A.p, piv.p);
            BEM_LAUNCH_CHECK();
            k_gj_pivot<<<div_up(n, 256), 256, 0, st>>>(n, p, A.p, piv.p, bad.p);
            BEM_LAUNCH_CHECK();
        }
        const size_t cnt = (size_t)n * n;
        k_bp_store<<<(unsigned)std::min<size_t>(div_up((int64_t)cnt, 256), 4096), 256, 0, st>>>(
            cnt, R, A.p, bp.inv64.p + bp.inv_off[k], bp.inv32.p + bp.inv_off[k]);
        BEM_LAUNCH_CHECK();
    }
    int hb = 0;
    BEM_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    BEM_CUDA(cudaStreamSynchronize(st));
    if (hb) fail(BEM_ERR_MESH, "bubble-block preconditioner: a bubble's single-layer block has a non-positive pivot");
    bp.ready = true;
}

}  // namespace

void block_precond_prepare(Context &c) {
    if (c.M < 1) fail(BEM_ERR_ARG, "the bubble-block preconditioner needs bubbles (vertex offsets)");
    if (!c.bp.ready) build(c);
    auto &bp = c.bp;
    for (size_t k = 0; k + 1 < bp.first.size(); ++k) {
        const int64_t nb = bp.first[k + 1] - bp.first[k];
        if (nb == 0) continue;
        k_bp_scales<<<(unsigned)nb, 128, 0, c.stream>>>(bp.nd[k], c.N, bp.bub_voff.p + bp.first[k], c.xyz.p,
                                                        bp.bub_scale.p + bp.first[k]);
        BEM_LAUNCH_CHECK();
    }
}

void block_precond_apply(Context &c, const double *y, double *z) {
    auto &bp = c.bp;
    const bool f64 = c.prm.precision == BEM_PREC_FP64;
    if (!f64) {  // the right-hand side in FP32 once, for every shape's product
        bp.yf.resize(c.N);
        k_to_f32<<<(unsigned)std::min<int64_t>(div_up(c.N, 256), 152 * 8), 256, 0, c.stream>>>(c.N, y, bp.yf.p);
        BEM_LAUNCH_CHECK();
    }
    for (size_t k = 0; k + 1 < bp.first.size(); ++k) {
        const int64_t nb = bp.first[k + 1] - bp.first[k];
        if (nb == 0) continue;
        const int n = bp.nd[k];
        const dim3 grid((unsigned)div_up(n, BP_TM), (unsigned)div_up(nb, BP_TN));
        const int64_t *vo = bp.bub_voff.p + bp.first[k];
        const double *sc = bp.bub_scale.p + bp.first[k];
        if (f64) {
            k_bp_apply<double><<<grid, BP_THREADS, 0, c.stream>>>(n, bp.inv64.p + bp.inv_off[k], (int)nb, vo, sc, y, z);
        } else {
            const dim3 gf((unsigned)div_up(n, BPF_TM), (unsigned)div_up(nb, BPF_TN));
            k_bp_apply_f32<<<gf, BPF_THREADS, 0, c.stream>>>(n, bp.inv32.p + bp.inv_off[k], (int)nb, vo, sc, bp.yf.p, z);
        }
        BEM_LAUNCH_CHECK();
    }
}

}  // namespace bem
