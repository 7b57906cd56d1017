// Learned GMRES initial guess (the paper's method starts from the previous step's q,
// Sections 3.5 and 3.8; that stays the fallback).
//
// Per bubble m, features f_m = [c(phi_m), c(q_prev,m), c(q_prev,m) - c(q_prev2,m)] with
// c(x) = G+ x the least-squares real spherical-harmonic coefficients of degree <= lmax on the
// bubble's initial directions (the projector of the shape filter, Eqs. (3.22)-(3.23)) and
// q_prev2 the start of the solve before. Samples are taken in the Adams-Bashforth phase, where
// consecutive solves are one step apart. A multilayer perceptron
//   h1 = relu(W1 f + b1), h2 = relu(W2 h1 + b2), h3 = relu(W3 h2 + b3), y = W4 h3 + b4
// predicts the change of q's coefficients from the solve's base start q_prev (the extrapolated
// guess when bem_step_params.guess >= 1, else the previous solve's q), and the guess is
// q0_m = q_prev,m + G_m y_m. Features and targets are scaled per column by their root mean
// square over the recorded samples (computed at training); training minimises the mean of
// |y - (c(q) - c(q_prev)) / tscale|^2 / 2 over recorded solves with Adam.
//
// The matrix products run on the tensor cores (tcgen05.mma kind::f16, BF16 operands, FP32
// accumulation in tensor memory); weights keep an FP32 master copy. Operands are loaded with
// arbitrary strides into the K-major core-matrix layout, which covers the transposed products
// of the backward pass. Waits on the MMA barrier are bounded.
#include "internal.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>

namespace bem {

struct Mlp {
    bool ready = false;
    int lmax = 10, Psh = 121;
    int dims[5] = {0, 0, 0, 0, 0};
    DevBuf<float> W[4], b[4], mW[4], vW[4], mb[4], vb[4], gW[4], gb[4];
    DevBuf<__nv_bfloat16> Wb[4];
    int64_t adam_t = 0;
    // recorded samples
    DevBuf<float> SF, ST;
    int64_t ns = 0, cap = 0;
    // work space (batch rows)
    int64_t wrows = 0;
    DevBuf<__nv_bfloat16> Hb[5];  // layer inputs in BF16 (Hb[0] = features)
    DevBuf<float> Z[4];           // pre-activations
    DevBuf<float> G;              // gradient w.r.t. a layer's output
    DevBuf<__nv_bfloat16> Gb;
    DevBuf<float> loss;
    ShBasis feat;
    DevBuf<double> qprev, cphi, cqp, cq, cqp_last;  // q_prev [N]; coefficients [M][Psh]
    bool have_last = false;
    bool uniform = false;  // the current solve is in the Adams-Bashforth phase
    bool record = false, use = false, compare = false;
    DevBuf<int> err;
    MlpStats stats;
    // input and output scales of the recorded data (per column: the root mean square over the
    // samples at the last training call; 1 before): the network sees features / fscale and is
    // trained on targets / tscale, and its output is multiplied by tscale in the guess
    DevBuf<float> fscale, tscale, Tb;
};

void mlp_free(Mlp *m) { delete m; }

namespace {

constexpr int GM = 128;           // tile rows
constexpr int GK = 64;            // K chunk (bf16): 128 bytes per row = 8 core matrices
constexpr int G_THREADS = 128;
constexpr uint32_t G_LBO = 128, G_SBO = 1024;
constexpr long long kWait = 1ll << 24;

__device__ __forceinline__ uint32_t sa(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ uint64_t desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((G_LBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((G_SBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, K-major.
constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity) {
    for (long long it = 0; it < kWait; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

enum { EPI_STORE = 0, EPI_BIAS_RELU = 1, EPI_BIAS = 2, EPI_RELU_MASK = 3 };

// C[m][n] = sum_k A(m,k) B(n,k), A(m,k) = A[m*sam + k*sak], B(n,k) = B[n*sbn + k*sbk].
// Epilogues: STORE: C = acc; BIAS: C = acc + bias[n]; BIAS_RELU: C = acc + bias[n] and
// H = bf16(relu(C)); RELU_MASK: C = acc where Zm[m*ldc + n] > 0, else 0 (and H = bf16(C)).
template <int NT>
__global__ void __launch_bounds__(G_THREADS) k_gemm_bf16(int M, int N, int K, const __nv_bfloat16 *__restrict__ A,
                                                         int64_t sam, int64_t sak, const __nv_bfloat16 *__restrict__ B,
                                                         int64_t sbn, int64_t sbk, float *__restrict__ C, int64_t ldc,
                                                         int epi, const float *__restrict__ bias,
                                                         const float *__restrict__ Zm, __nv_bfloat16 *__restrict__ H,
                                                         int *__restrict__ err) {
    __shared__ __align__(1024) __nv_bfloat16 As[GM * GK];
    __shared__ __align__(1024) __nv_bfloat16 Bs[NT * GK];
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * GM, n0 = blockIdx.y * NT;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sa(&bar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(&tslot)), "r"(NT));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tslot;
    uint32_t phase = 0;
    bool ok = true;
    const int nchunk = (K + GK - 1) / GK;
    for (int kc = 0; kc < nchunk && ok; ++kc) {
        // stage: 16-byte units (8 consecutive k of one row) in the canonical layout
        for (int u = tid; u < (GM + NT) * (GK / 8); u += G_THREADS) {
            const bool isA = u < GM * (GK / 8);
            const int uu = isA ? u : u - GM * (GK / 8);
            const int row = uu / (GK / 8), j = uu % (GK / 8);
            __nv_bfloat16 v[8];
            const int k0 = kc * GK + j * 8;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int k = k0 + e;
                __nv_bfloat16 x = __float2bfloat16(0.f);
                if (isA) {
                    const int m = m0 + row;
                    if (m < M && k < K) x = A[(int64_t)m * sam + (int64_t)k * sak];
                } else {
                    const int n = n0 + row;
                    if (n < N && k < K) x = B[(int64_t)n * sbn + (int64_t)k * sbk];
                }
                v[e] = x;
            }
            __nv_bfloat16 *dst = (isA ? As : Bs) + (row / 8) * 512 + j * 64 + (row % 8) * 8;  // elements
            *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(v);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int ksteps = (min(GK, K - kc * GK) + 15) / 16;
            for (int s = 0; s < ksteps; ++s) {
                const uint32_t o = s * 2 * G_LBO;
                const uint32_t acc = (kc > 0 || s > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                    "l"(desc(sa(As) + o)), "l"(desc(sa(Bs) + o)), "r"(idesc_bf16(GM, NT)), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sa(&bar))
                         : "memory");
        }
        __syncwarp();
        const int bad = __syncthreads_or(wait_bar(sa(&bar), phase) ? 0 : 1);
        if (bad) {
            wait_bar(sa(&bar), phase);
            if (tid == 0) atomicOr(err, 1);
            ok = false;
        }
        phase ^= 1u;
        __syncthreads();
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
        const int m = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < NT; c0 += 16) {
            uint32_t v[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (m < M) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int n = n0 + c0 + i;
                    if (n >= N) continue;
                    float a = __uint_as_float(v[i]);
                    const int64_t ix = (int64_t)m * ldc + n;
                    if (epi == EPI_BIAS || epi == EPI_BIAS_RELU) a += bias[n];
                    if (epi == EPI_RELU_MASK) a = Zm[ix] > 0.f ? a : 0.f;
                    C[ix] = a;
                    if (epi == EPI_BIAS_RELU) H[ix] = __float2bfloat16(fmaxf(a, 0.f));
                    if (epi == EPI_RELU_MASK && H) H[ix] = __float2bfloat16(a);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NT));
}

__global__ void k_f2bf(int64_t n, const float *__restrict__ x, __nv_bfloat16 *__restrict__ y) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16(x[i]);
}

__global__ void k_d2bf(int64_t n, const double *__restrict__ x, __nv_bfloat16 *__restrict__ y) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16((float)x[i]);
}

// G = (Y - T) / B (also bf16), loss partial sums per block
__global__ void k_loss_grad(int64_t n, int B, const float *__restrict__ Y, const float *__restrict__ T,
                            float *__restrict__ G, __nv_bfloat16 *__restrict__ Gb, float *__restrict__ loss) {
    __shared__ float red[256];
    float s = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float d = Y[i] - T[i];
        s += d * d;
        float g = d / (float)B;
        G[i] = g;
        Gb[i] = __float2bfloat16(g);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, 0.5f * red[0] / (float)B);
}

// db[n] = sum_rows G[row][n]
__global__ void k_colsum(int rows, int cols, const float *__restrict__ G, float *__restrict__ db) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= cols) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += G[(int64_t)r * cols + n];
    db[n] = s;
}

__global__ void k_adam(int64_t n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float c1, float c2, float eps,
                       __nv_bfloat16 *__restrict__ pb) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float mm = b1 * m[i] + (1.f - b1) * g[i];
    float vv = b2 * v[i] + (1.f - b2) * g[i] * g[i];
    m[i] = mm;
    v[i] = vv;
    float x = p[i] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    p[i] = x;
    if (pb) pb[i] = __float2bfloat16(x);
}

// out[m][p] = sum_i Gp_m[p][i] x[a_m + i]  (per-bubble SH coefficients; one block per bubble)
__global__ void k_sh_project(int64_t M, const int64_t *__restrict__ voff, const int32_t *__restrict__ shape_of,
                             const int64_t *__restrict__ g_off, int P, const double *__restrict__ Gp,
                             const double *__restrict__ x, double *__restrict__ out) {
    int m = blockIdx.x;
    int64_t a = voff[m];
    int nd = (int)(voff[m + 1] - a);
    const double *G = Gp + g_off[shape_of[m]];
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < nd; ++i) s = fma(G[(size_t)p * nd + i], x[a + i], s);
        out[(size_t)m * P + p] = s;
    }
}

// q[a_m + i] = qprev[a_m + i] + sum_p G_m[i][p] y[m][p]
__global__ void k_sh_synth_add(int64_t M, const int64_t *__restrict__ voff, const int32_t *__restrict__ shape_of,
                               const int64_t *__restrict__ g_off, int P, const double *__restrict__ G,
                               const float *__restrict__ y, const float *__restrict__ yscale,
                               const double *__restrict__ qprev, double *__restrict__ q) {
    int m = blockIdx.x;
    int64_t a = voff[m];
    int nd = (int)(voff[m + 1] - a);
    const double *Gm = G + g_off[shape_of[m]];
    for (int i = threadIdx.x; i < nd; i += blockDim.x) {
        double s = qprev[a + i];
        for (int p = 0; p < P; ++p)
            s = fma(Gm[(size_t)i * P + p], (double)y[(size_t)m * P + p] * (double)yscale[p], s);
        q[a + i] = s;
    }
}

// per column: out[j] = sqrt(mean_r X[r][j]^2) (1 where that is 0); one thread per column
__global__ void k_col_rms(int64_t rows, int cols, const float *__restrict__ X, float *__restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    double s = 0.0;
    for (int64_t r = 0; r < rows; ++r) {
        const double v = X[r * cols + j];
        s += v * v;
    }
    const double rms = sqrt(s / (double)(rows > 0 ? rows : 1));
    out[j] = rms > 0.0 ? (float)rms : 1.f;
}

// y[r][j] = bf16(x[r][j] / scale[j]) for the network input
__global__ void k_f2bf_scaled(int64_t n, int cols, const float *__restrict__ x, const float *__restrict__ scale,
                              __nv_bfloat16 *__restrict__ y) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16(x[i] / scale[i % cols]);
}

// y[r][j] = x[r][j] / scale[j] (training targets)
__global__ void k_div_cols(int64_t n, int cols, const float *__restrict__ x, const float *__restrict__ scale,
                           float *__restrict__ y) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = x[i] / scale[i % cols];
}

// features [M][3P] (float): c(phi), c(q_prev), c(q_prev) - c(q_prev2); targets [M][P] = c(q) - c(q_prev)
__global__ void k_pack_features(int64_t M, int P, const double *__restrict__ cphi, const double *__restrict__ cqp,
                                const double *__restrict__ cqp_last, float *__restrict__ F) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= M * 3 * P) return;
    int64_t m = e / (3 * P);
    int k = (int)(e % (3 * P));
    double v;
    if (k < P) v = cphi[m * P + k];
    else if (k < 2 * P) v = cqp[m * P + (k - P)];
    else v = cqp_last ? cqp[m * P + (k - 2 * P)] - cqp_last[m * P + (k - 2 * P)] : 0.0;
    F[e] = (float)v;
}

__global__ void k_pack_targets(int64_t M, int P, const double *__restrict__ cq, const double *__restrict__ cqp,
                               float *__restrict__ T) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= M * P) return;
    T[e] = (float)(cq[e] - cqp[e]);
}

Mlp &mlp_of(Context &c) {
    if (!c.mlp) c.mlp = new Mlp();
    return *c.mlp;
}

void gemm(Context &c, Mlp &m, int M, int N, int K, const __nv_bfloat16 *A, int64_t sam, int64_t sak,
          const __nv_bfloat16 *B, int64_t sbn, int64_t sbk, float *C, int64_t ldc, int epi, const float *bias,
          const float *Zm, __nv_bfloat16 *H) {
    if (N > 128) {
        dim3 grid((M + GM - 1) / GM, (N + 255) / 256);
        k_gemm_bf16<256><<<grid, G_THREADS, 0, c.stream>>>(M, N, K, A, sam, sak, B, sbn, sbk, C, ldc, epi, bias, Zm, H,
                                                          m.err.p);
    } else {
        dim3 grid((M + GM - 1) / GM, (N + 127) / 128);
        k_gemm_bf16<128><<<grid, G_THREADS, 0, c.stream>>>(M, N, K, A, sam, sak, B, sbn, sbk, C, ldc, epi, bias, Zm, H,
                                                          m.err.p);
    }
    BEM_LAUNCH_CHECK();
}

void ensure_work(Mlp &m, int64_t rows) {
    if (rows <= m.wrows) return;
    m.wrows = rows;
    for (int i = 0; i <= 4; ++i) m.Hb[i].resize((size_t)rows * m.dims[i]);
    for (int i = 0; i < 4; ++i) m.Z[i].resize((size_t)rows * m.dims[i + 1]);
    int dmax = *std::max_element(m.dims, m.dims + 5);
    m.G.resize((size_t)rows * dmax);
    m.Gb.resize((size_t)rows * dmax);
}

// Forward pass on Hb[0] (rows x dims[0]); Z[3] holds the output y.
void forward(Context &c, Mlp &m, int rows) {
    for (int i = 0; i < 4; ++i) {
        const bool last = i == 3;
        gemm(c, m, rows, m.dims[i + 1], m.dims[i], m.Hb[i].p, m.dims[i], 1, m.Wb[i].p, m.dims[i], 1, m.Z[i].p,
             m.dims[i + 1], last ? EPI_BIAS : EPI_BIAS_RELU, m.b[i].p, nullptr, last ? nullptr : m.Hb[i + 1].p);
    }
}

// Loss and gradients (into gW, gb) for targets T (rows x dims[4], float). Returns loss on device.
void backward(Context &c, Mlp &m, int rows, const float *T) {
    const int tb = 256;
    BEM_CUDA(cudaMemsetAsync(m.loss.p, 0, sizeof(float), c.stream));
    int64_t no = (int64_t)rows * m.dims[4];
    k_loss_grad<<<std::min<int64_t>(div_up(no, tb), 512), tb, 0, c.stream>>>(no, rows, m.Z[3].p, T, m.G.p, m.Gb.p,
                                                                              m.loss.p);
    BEM_LAUNCH_CHECK();
    for (int i = 3; i >= 0; --i) {
        const int dout = m.dims[i + 1], din = m.dims[i];
        // dW_i = G^T H_i  [dout x din]: A(o, r) = G[r*dout + o], B(k, r) = H_i[r*din + k]
        gemm(c, m, dout, din, rows, m.Gb.p, 1, dout, m.Hb[i].p, 1, din, m.gW[i].p, din, EPI_STORE, nullptr, nullptr,
             nullptr);
        k_colsum<<<div_up(dout, 128), 128, 0, c.stream>>>(rows, dout, m.G.p, m.gb[i].p);
        BEM_LAUNCH_CHECK();
        if (i > 0) {
            // G_prev = (G W_i) masked by Z_{i-1} > 0: A(r, o) = G[r*dout + o], B(k, o) = W_i[o*din + k]
            gemm(c, m, rows, din, dout, m.Gb.p, dout, 1, m.Wb[i].p, 1, din, m.G.p, din, EPI_RELU_MASK, nullptr,
                 m.Z[i - 1].p, m.Gb.p);
        }
    }
}

void check_err(Context &c, Mlp &m) {
    int h = 0;
    BEM_CUDA(cudaMemcpyAsync(&h, m.err.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    BEM_CUDA(cudaStreamSynchronize(c.stream));
    if (h) fail(BEM_ERR_TIMEOUT, "tensor-core GEMM wait ran out");
}

}  // namespace

int64_t mlp_num_params(const Mlp &m) {
    int64_t n = 0;
    for (int i = 0; i < 4; ++i) n += (int64_t)m.dims[i + 1] * m.dims[i] + m.dims[i + 1];
    return n;
}

void mlp_init(Context &c, int hidden, int lmax, uint64_t seed, const double *xyz0) {
    if (hidden < 16 || hidden > 256 || hidden % 16) fail(BEM_ERR_ARG, "hidden width must be a multiple of 16 in 16..256");
    if (lmax < 0 || lmax > 10) fail(BEM_ERR_ARG, "lmax must be in 0..10");
    Mlp &m = mlp_of(c);
    m.lmax = lmax;
    m.Psh = (lmax + 1) * (lmax + 1);
    const int dims[5] = {3 * m.Psh, hidden, hidden, hidden, m.Psh};
    std::memcpy(m.dims, dims, sizeof(dims));
    m.err.resize(1);
    m.loss.resize(1);
    BEM_CUDA(cudaMemsetAsync(m.err.p, 0, sizeof(int), c.stream));
    std::mt19937_64 rng(seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    for (int i = 0; i < 4; ++i) {
        const int64_t nw = (int64_t)dims[i + 1] * dims[i];
        std::vector<float> w(nw), bz(dims[i + 1], 0.f);
        const double sc = std::sqrt(2.0 / dims[i]) * (i == 3 ? 0.1 : 1.0);
        for (auto &x : w) x = (float)(nd(rng) * sc);
        for (auto *bf : {&m.W[i], &m.mW[i], &m.vW[i], &m.gW[i]}) bf->resize(nw);
        for (auto *bf : {&m.b[i], &m.mb[i], &m.vb[i], &m.gb[i]}) bf->resize(dims[i + 1]);
        m.Wb[i].resize(nw);
        BEM_CUDA(cudaMemcpyAsync(m.W[i].p, w.data(), nw * sizeof(float), cudaMemcpyHostToDevice, c.stream));
        BEM_CUDA(cudaMemcpyAsync(m.b[i].p, bz.data(), bz.size() * sizeof(float), cudaMemcpyHostToDevice, c.stream));
        BEM_CUDA(cudaMemsetAsync(m.mW[i].p, 0, nw * sizeof(float), c.stream));
        BEM_CUDA(cudaMemsetAsync(m.vW[i].p, 0, nw * sizeof(float), c.stream));
        BEM_CUDA(cudaMemsetAsync(m.mb[i].p, 0, dims[i + 1] * sizeof(float), c.stream));
        BEM_CUDA(cudaMemsetAsync(m.vb[i].p, 0, dims[i + 1] * sizeof(float), c.stream));
        k_f2bf<<<div_up(nw, 256), 256, 0, c.stream>>>(nw, m.W[i].p, m.Wb[i].p);
        BEM_LAUNCH_CHECK();
        BEM_CUDA(cudaStreamSynchronize(c.stream));  // host vectors go out of scope
    }
    m.adam_t = 0;
    m.ns = 0;
    m.wrows = 0;
    m.have_last = false;
    {
        std::vector<float> one(std::max(dims[0], dims[4]), 1.f);
        m.fscale.resize(dims[0]);
        m.tscale.resize(dims[4]);
        BEM_CUDA(cudaMemcpyAsync(m.fscale.p, one.data(), dims[0] * sizeof(float), cudaMemcpyHostToDevice, c.stream));
        BEM_CUDA(cudaMemcpyAsync(m.tscale.p, one.data(), dims[4] * sizeof(float), cudaMemcpyHostToDevice, c.stream));
        BEM_CUDA(cudaStreamSynchronize(c.stream));
    }
    // features basis from the initial shapes
    DevBuf<int> bad;
    bad.resize(1);
    BEM_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), c.stream));
    build_sh_basis(c, lmax + 1, m.feat, bad.p, xyz0);
    int hb = 0;
    BEM_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    BEM_CUDA(cudaStreamSynchronize(c.stream));
    if (hb) fail(BEM_ERR_MESH, "singular spherical-harmonic basis for the features");
    m.ready = true;
}

void mlp_set_mode(Context &c, int record, int use, int compare) {
    Mlp &m = mlp_of(c);
    if (!m.ready) fail(BEM_ERR_NOT_BUILT, "bem_mlp_init has not been called");
    m.record = record != 0;
    m.use = use != 0;
    m.compare = compare != 0;
}

bool mlp_active(Context &c) { return c.mlp && c.mlp->ready && (c.mlp->record || c.mlp->use); }
bool mlp_compare(Context &c) { return c.mlp && c.mlp->ready && c.mlp->use && c.mlp->compare && c.mlp->uniform; }

// Before a solve with initial guess q (= q_prev): features; when the solve is in the uniform
// (Adams-Bashforth) phase, record them and, with `use`, replace q by q_prev + G y.
void mlp_before_solve(Context &c, const double *phi, double *q, bool uniform) {
    Mlp &m = *c.mlp;
    const int64_t M = c.M, N = c.N;
    const int P = m.Psh;
    m.uniform = uniform;
    m.qprev.resize(N);
    m.cphi.resize((size_t)M * P);
    m.cqp.resize((size_t)M * P);
    m.cq.resize((size_t)M * P);
    m.cqp_last.resize((size_t)M * P);
    BEM_CUDA(cudaMemcpyAsync(m.qprev.p, q, N * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    DevBuf<int64_t> &voff = c.voff_d;
    k_sh_project<<<(unsigned)M, 128, 0, c.stream>>>(M, voff.p, m.feat.shape_of.p, m.feat.g_off.p, P, m.feat.Gp.p, phi,
                                                    m.cphi.p);
    k_sh_project<<<(unsigned)M, 128, 0, c.stream>>>(M, voff.p, m.feat.shape_of.p, m.feat.g_off.p, P, m.feat.Gp.p, q,
                                                    m.cqp.p);
    BEM_LAUNCH_CHECK();
    ensure_work(m, M);
    DevBuf<float> F;
    F.resize((size_t)M * 3 * P);
    k_pack_features<<<div_up(M * 3 * P, 256), 256, 0, c.stream>>>(M, P, m.cphi.p, m.cqp.p,
                                                                  m.have_last ? m.cqp_last.p : nullptr, F.p);
    BEM_LAUNCH_CHECK();
    BEM_CUDA(cudaMemcpyAsync(m.cqp_last.p, m.cqp.p, M * P * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    m.have_last = true;
    if (m.record && uniform) {
        if (m.ns + M > m.cap) {
            int64_t nc = std::max<int64_t>(2 * m.cap, m.ns + M);
            DevBuf<float> nf, nt;
            nf.resize((size_t)nc * 3 * P);
            nt.resize((size_t)nc * P);
            if (m.ns) {
                BEM_CUDA(cudaMemcpyAsync(nf.p, m.SF.p, m.ns * 3 * P * sizeof(float), cudaMemcpyDeviceToDevice, c.stream));
                BEM_CUDA(cudaMemcpyAsync(nt.p, m.ST.p, m.ns * P * sizeof(float), cudaMemcpyDeviceToDevice, c.stream));
            }
            BEM_CUDA(cudaStreamSynchronize(c.stream));
            std::swap(m.SF.p, nf.p);
            std::swap(m.SF.cap, nf.cap);
            std::swap(m.SF.n, nf.n);
            std::swap(m.ST.p, nt.p);
            std::swap(m.ST.cap, nt.cap);
            std::swap(m.ST.n, nt.n);
            m.cap = nc;
        }
        BEM_CUDA(cudaMemcpyAsync(m.SF.p + m.ns * 3 * P, F.p, M * 3 * P * sizeof(float), cudaMemcpyDeviceToDevice,
                                 c.stream));
    }
    if (m.use && uniform) {
        k_f2bf_scaled<<<div_up(M * 3 * P, 256), 256, 0, c.stream>>>(M * 3 * P, 3 * P, F.p, m.fscale.p, m.Hb[0].p);
        BEM_LAUNCH_CHECK();
        forward(c, m, (int)M);
        k_sh_synth_add<<<(unsigned)M, 128, 0, c.stream>>>(M, voff.p, m.feat.shape_of.p, m.feat.g_off.p, P, m.feat.G.p,
                                                          m.Z[3].p, m.tscale.p, m.qprev.p, q);
        BEM_LAUNCH_CHECK();
    }
    BEM_CUDA(cudaStreamSynchronize(c.stream));
}

const double *mlp_qprev(Context &c) { return c.mlp->qprev.p; }

// After the solve: with `record`, the target c(q) - c(q_prev) of the sample stored before.
void mlp_after_solve(Context &c, const double *q) {
    Mlp &m = *c.mlp;
    if (!m.record || !m.uniform) return;
    const int64_t M = c.M;
    const int P = m.Psh;
    DevBuf<int64_t> &voff = c.voff_d;
    k_sh_project<<<(unsigned)M, 128, 0, c.stream>>>(M, voff.p, m.feat.shape_of.p, m.feat.g_off.p, P, m.feat.Gp.p, q,
                                                    m.cq.p);
    BEM_LAUNCH_CHECK();
    k_pack_targets<<<div_up(M * P, 256), 256, 0, c.stream>>>(M, P, m.cq.p, m.cqp.p, m.ST.p + m.ns * P);
    BEM_LAUNCH_CHECK();
    m.ns += M;
}

// Adam over the recorded samples in minibatches of `batch` rows, `epochs` passes; returns the
// mean loss of the last epoch.
double mlp_train(Context &c, int epochs, int batch, double lr) {
    Mlp &m = mlp_of(c);
    if (!m.ready) fail(BEM_ERR_NOT_BUILT, "bem_mlp_init has not been called");
    if (m.ns == 0) fail(BEM_ERR_ARG, "no recorded samples");
    batch = (int)std::min<int64_t>(std::max(1, batch), m.ns);
    ensure_work(m, batch);
    const int P = m.Psh;
    // column scales of the recorded features and targets (the network learns the scaled map)
    k_col_rms<<<div_up(3 * P, 128), 128, 0, c.stream>>>(m.ns, 3 * P, m.SF.p, m.fscale.p);
    k_col_rms<<<div_up(P, 128), 128, 0, c.stream>>>(m.ns, P, m.ST.p, m.tscale.p);
    BEM_LAUNCH_CHECK();
    m.Tb.resize((size_t)batch * P);
    double last = 0.0;
    for (int ep = 0; ep < epochs; ++ep) {
        double tot = 0.0;
        int nb = 0;
        for (int64_t r0 = 0; r0 < m.ns; r0 += batch) {
            const int rows = (int)std::min<int64_t>(batch, m.ns - r0);
            k_f2bf_scaled<<<div_up((int64_t)rows * 3 * P, 256), 256, 0, c.stream>>>(
                (int64_t)rows * 3 * P, 3 * P, m.SF.p + r0 * 3 * P, m.fscale.p, m.Hb[0].p);
            k_div_cols<<<div_up((int64_t)rows * P, 256), 256, 0, c.stream>>>((int64_t)rows * P, P, m.ST.p + r0 * P,
                                                                             m.tscale.p, m.Tb.p);
            BEM_LAUNCH_CHECK();
            forward(c, m, rows);
            backward(c, m, rows, m.Tb.p);
            m.adam_t += 1;
            const float b1 = 0.9f, b2 = 0.999f;
            const float c1 = 1.f - std::pow(b1, (float)m.adam_t), c2 = 1.f - std::pow(b2, (float)m.adam_t);
            for (int i = 0; i < 4; ++i) {
                int64_t nw = (int64_t)m.dims[i + 1] * m.dims[i];
                k_adam<<<div_up(nw, 256), 256, 0, c.stream>>>(nw, m.W[i].p, m.gW[i].p, m.mW[i].p, m.vW[i].p, (float)lr,
                                                               b1, b2, c1, c2, 1e-8f, m.Wb[i].p);
                k_adam<<<div_up(m.dims[i + 1], 256), 256, 0, c.stream>>>(m.dims[i + 1], m.b[i].p, m.gb[i].p, m.mb[i].p,
                                                                          m.vb[i].p, (float)lr, b1, b2, c1, c2, 1e-8f,
                                                                          nullptr);
                BEM_LAUNCH_CHECK();
            }
            float h = 0.f;
            BEM_CUDA(cudaMemcpyAsync(&h, m.loss.p, sizeof(float), cudaMemcpyDeviceToHost, c.stream));
            BEM_CUDA(cudaStreamSynchronize(c.stream));
            tot += h;
            ++nb;
        }
        last = tot / std::max(1, nb);
    }
    check_err(c, m);
    return last;
}

// Loss and flat gradients (W1, b1, ..., W4, b4; W row-major [out][in]) for one batch given in
// FP64 host or device arrays already copied to device (F [B][din], T [B][dout]).
double mlp_loss_grad(Context &c, int B, const double *F, const double *T, double *grads_dev) {
    Mlp &m = mlp_of(c);
    if (!m.ready) fail(BEM_ERR_NOT_BUILT, "bem_mlp_init has not been called");
    ensure_work(m, B);
    const int din = m.dims[0], dout = m.dims[4];
    k_d2bf<<<div_up((int64_t)B * din, 256), 256, 0, c.stream>>>((int64_t)B * din, F, m.Hb[0].p);
    BEM_LAUNCH_CHECK();
    DevBuf<float> Tf;
    Tf.resize((size_t)B * dout);
    std::vector<double> th((size_t)B * dout);
    BEM_CUDA(cudaMemcpyAsync(th.data(), T, th.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    BEM_CUDA(cudaStreamSynchronize(c.stream));
    std::vector<float> tf(th.begin(), th.end());
    BEM_CUDA(cudaMemcpyAsync(Tf.p, tf.data(), tf.size() * sizeof(float), cudaMemcpyHostToDevice, c.stream));
    forward(c, m, B);
    backward(c, m, B, Tf.p);
    float h = 0.f;
    BEM_CUDA(cudaMemcpyAsync(&h, m.loss.p, sizeof(float), cudaMemcpyDeviceToHost, c.stream));
    int64_t off = 0;
    for (int i = 0; i < 4; ++i) {
        int64_t nw = (int64_t)m.dims[i + 1] * m.dims[i];
        std::vector<float> a(nw), bb(m.dims[i + 1]);
        BEM_CUDA(cudaMemcpyAsync(a.data(), m.gW[i].p, nw * sizeof(float), cudaMemcpyDeviceToHost, c.stream));
        BEM_CUDA(cudaMemcpyAsync(bb.data(), m.gb[i].p, bb.size() * sizeof(float), cudaMemcpyDeviceToHost, c.stream));
        BEM_CUDA(cudaStreamSynchronize(c.stream));
        std::vector<double> ad(a.begin(), a.end()), bd(bb.begin(), bb.end());
        BEM_CUDA(cudaMemcpyAsync(grads_dev + off, ad.data(), nw * sizeof(double), cudaMemcpyHostToDevice, c.stream));
        off += nw;
        BEM_CUDA(cudaMemcpyAsync(grads_dev + off, bd.data(), bd.size() * sizeof(double), cudaMemcpyHostToDevice,
                                 c.stream));
        off += m.dims[i + 1];
        BEM_CUDA(cudaStreamSynchronize(c.stream));
    }
    check_err(c, m);
    return h;
}

// Forward only: Y [B][dout] (device FP64) from F [B][din] (device FP64).
void mlp_forward(Context &c, int B, const double *F, double *Y) {
    Mlp &m = mlp_of(c);
    if (!m.ready) fail(BEM_ERR_NOT_BUILT, "bem_mlp_init has not been called");
    ensure_work(m, B);
    const int din = m.dims[0], dout = m.dims[4];
    k_d2bf<<<div_up((int64_t)B * din, 256), 256, 0, c.stream>>>((int64_t)B * din, F, m.Hb[0].p);
    BEM_LAUNCH_CHECK();
    forward(c, m, B);
    std::vector<float> y((size_t)B * dout);
    BEM_CUDA(cudaMemcpyAsync(y.data(), m.Z[3].p, y.size() * sizeof(float), cudaMemcpyDeviceToHost, c.stream));
    BEM_CUDA(cudaStreamSynchronize(c.stream));
    std::vector<double> yd(y.begin(), y.end());
    BEM_CUDA(cudaMemcpyAsync(Y, yd.data(), yd.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream));
    BEM_CUDA(cudaStreamSynchronize(c.stream));
    check_err(c, m);
}

// Flat FP64 parameter vector in the order W1, b1, ..., W4, b4 (host memory).
void mlp_get_params(Context &c, double *out) {
    Mlp &m = mlp_of(c);
    if (!m.ready) fail(BEM_ERR_NOT_BUILT, "bem_mlp_init has not been called");
    int64_t off = 0;
    for (int i = 0; i < 4; ++i) {
        int64_t nw = (int64_t)m.dims[i + 1] * m.dims[i];
        std::vector<float> a(nw), bb(m.dims[i + 1]);
        BEM_CUDA(cudaMemcpyAsync(a.data(), m.W[i].p, nw * sizeof(float), cudaMemcpyDeviceToHost, c.stream));
        BEM_CUDA(cudaMemcpyAsync(bb.data(), m.b[i].p, bb.size() * sizeof(float), cudaMemcpyDeviceToHost, c.stream));
        BEM_CUDA(cudaStreamSynchronize(c.stream));
        for (int64_t k = 0; k < nw; ++k) out[off++] = a[k];
        for (float v : bb) out[off++] = v;
    }
}

void mlp_set_params(Context &c, const double *in) {
    Mlp &m = mlp_of(c);
    if (!m.ready) fail(BEM_ERR_NOT_BUILT, "bem_mlp_init has not been called");
    int64_t off = 0;
    for (int i = 0; i < 4; ++i) {
        int64_t nw = (int64_t)m.dims[i + 1] * m.dims[i];
        std::vector<float> a(in + off, in + off + nw);
        off += nw;
        std::vector<float> bb(in + off, in + off + m.dims[i + 1]);
        off += m.dims[i + 1];
        BEM_CUDA(cudaMemcpyAsync(m.W[i].p, a.data(), nw * sizeof(float), cudaMemcpyHostToDevice, c.stream));
        BEM_CUDA(cudaMemcpyAsync(m.b[i].p, bb.data(), bb.size() * sizeof(float), cudaMemcpyHostToDevice, c.stream));
        k_f2bf<<<div_up(nw, 256), 256, 0, c.stream>>>(nw, m.W[i].p, m.Wb[i].p);
        BEM_LAUNCH_CHECK();
        BEM_CUDA(cudaStreamSynchronize(c.stream));
    }
}

int64_t mlp_samples(Context &c) { return c.mlp ? c.mlp->ns : 0; }
MlpStats &mlp_stats(Context &c) { return mlp_of(c).stats; }
const int *mlp_dims(Context &c) { return mlp_of(c).dims; }

}  // namespace bem
