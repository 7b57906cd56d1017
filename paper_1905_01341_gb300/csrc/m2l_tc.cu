// M2L translations on the 5th-generation tensor cores (tcgen05, TMEM accumulators).
//
// For one offset class c and a chunk of up to 128/R (source, target) pairs, the product
//   Y[pair, rhs][n] = sum_k T_c[n][k] X[src, rhs][k]
// is one MMA tile D = A B^T with M = 128 rows (pair, rhs), N = P rounded up to 16 output
// coefficients and K = P input coefficients: A = the gathered multipole rows, B = T_c (row n of
// T_c is K-contiguous, i.e. K-major). Accuracy: both operands are split into three TF32 pieces,
// x = x0 + x1 + x2 (x0 = tf32(x), x1 = tf32(x - x0), x2 = the rest), and D accumulates the six
// products x0 y0 + x0 y1 + x1 y0 + x0 y2 + x1 y1 + x2 y0 in FP32; the dropped terms are ~2^-33
// of the product, so the translation is as accurate as an FP32 product. (Translation sums
// cancel strongly, so a two-piece split, ~2^-21 per product, leaves noise near 1e-6 in the
// operator, which a GMRES solve to 1e-6 cannot tolerate.)
//
// Operands are staged through shared memory in the canonical K-major layout without swizzle:
// 8-row x 16-byte core matrices, core matrices adjacent in K are 128 B apart (leading byte
// offset) and 8-row groups are 1024 B apart (stride byte offset) within a 32-wide K chunk.
// One elected thread issues the MMAs; completion is signalled through an mbarrier whose
// waits are bounded: a wait that runs out sets an error flag and the block skips ahead,
// releasing its tensor memory.
#include "internal.h"

namespace bem {
namespace {

constexpr int TC_M = 128;          // rows per tile
constexpr int TC_KC = 32;          // K chunk staged per round
constexpr int TC_THREADS = 128;
constexpr int TC_KGROUPS = TC_KC / 4;  // 16-byte core-matrix columns per chunk
constexpr uint32_t TC_LBO = 128;       // bytes between K-adjacent core matrices
constexpr uint32_t TC_SBO = 128 * TC_KGROUPS;  // bytes between 8-row groups (1024)
constexpr long long kWaitLimit = 1ll << 24;    // iterations before a wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((TC_LBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((TC_SBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for this architecture; no swizzle, base offset 0
    return d;
}

// kind::tf32 instruction descriptor: D = F32, A = B = TF32, both K-major, N and M given.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float tf32_head(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// x = x0 + x1 + x2 with x0, x1 TF32-representable (x2 is truncated to TF32 by the MMA).
__device__ __forceinline__ void split3(float4 v, float4 &x0, float4 &x1, float4 &x2) {
    x0 = make_float4(tf32_head(v.x), tf32_head(v.y), tf32_head(v.z), tf32_head(v.w));
    float4 r = make_float4(v.x - x0.x, v.y - x0.y, v.z - x0.z, v.w - x0.w);
    x1 = make_float4(tf32_head(r.x), tf32_head(r.y), tf32_head(r.z), tf32_head(r.w));
    x2 = make_float4(r.x - x1.x, r.y - x1.y, r.z - x1.z, r.w - x1.w);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (long long it = 0; it < kWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Row-major T_c [P][P] (FP32) -> per class, per K chunk, an N_pad x 32 block in the canonical
// K-major core-matrix layout, zero-padded (n >= P or k >= P).
__global__ void k_build_tc_table(int P, int Npad, int Kpad, const float *__restrict__ T, float *__restrict__ out) {
    const int cls = blockIdx.y;
    const size_t block = (size_t)Npad * TC_KC;
    const int nchunk = Kpad / TC_KC;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < block * nchunk;
         e += (size_t)gridDim.x * blockDim.x) {
        int kc = (int)(e / block);
        int rem = (int)(e % block);
        // inverse of the canonical offset: rem = (n/8)*256 + (kk/4)*32 + (n%8)*4 + kk%4
        int g = rem / 256, r2 = rem % 256;
        int j = r2 / 32, r3 = r2 % 32;
        int n = g * 8 + r3 / 4, kk = j * 4 + r3 % 4;
        int k = kc * TC_KC + kk;
        float v = (n < P && k < P) ? T[((size_t)cls * P + n) * P + k] : 0.f;
        out[(size_t)cls * block * nchunk + e] = v;
    }
}

template <int R>
__global__ void __launch_bounds__(TC_THREADS) k_m2l_tc(int P, int Npad, int Kpad, const float *__restrict__ tcB,
                                                       const XChunk *__restrict__ chunks,
                                                       const int32_t *__restrict__ srcs,
                                                       const float *__restrict__ X, float *__restrict__ Ypair,
                                                       int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    // layout: A0, A1, A2 [128 x 32] each, B0, B1, B2 [Npad x 32] each, then barrier + tmem slot
    float *A0 = reinterpret_cast<float *>(smem);
    float *A1 = A0 + TC_M * TC_KC;
    float *A2 = A1 + TC_M * TC_KC;
    float *B0 = A2 + TC_M * TC_KC;
    float *B1 = B0 + Npad * TC_KC;
    float *B2 = B1 + Npad * TC_KC;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(B2 + Npad * TC_KC);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mbar + 1);
    __shared__ int s_src[TC_M];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const XChunk ch = chunks[blockIdx.x];
    const int nrows = ch.count * R;
    if (tid < TC_M) s_src[tid] = (tid < nrows) ? srcs[ch.start + tid / R] : -1;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = make_idesc(TC_M, Npad);
    const int nchunk = Kpad / TC_KC;
    const size_t bblock = (size_t)Npad * TC_KC;
    const float *Bc = tcB + (size_t)ch.cls * bblock * nchunk;
    uint32_t phase = 0;
    bool ok = true;

    for (int kc = 0; kc < nchunk && ok; ++kc) {
        // A: thread -> (row within an 8-row group, 16-byte K column); rows = 2 groups per pass
        {
            const int t64 = tid & 63, r8 = t64 & 7, j = t64 >> 3;
            const int k0 = kc * TC_KC + j * 4;
            for (int gp = (tid >> 6); gp < TC_M / 8; gp += 2) {
                const int row = gp * 8 + r8;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                const int s = s_src[row];
                if (s >= 0 && k0 < P) {
                    const float *src = X + ((size_t)s * R + (row % R)) * P + k0;
                    v = *reinterpret_cast<const float4 *>(src);  // P % 4 == 0, k0 % 4 == 0
                }
                float4 x0, x1, x2;
                split3(v, x0, x1, x2);
                const int off = gp * 256 + j * 32 + r8 * 4;  // floats
                *reinterpret_cast<float4 *>(A0 + off) = x0;
                *reinterpret_cast<float4 *>(A1 + off) = x1;
                *reinterpret_cast<float4 *>(A2 + off) = x2;
            }
        }
        // B: linear copy of the pre-tiled chunk block, split on the way
        {
            const float4 *src = reinterpret_cast<const float4 *>(Bc + (size_t)kc * bblock);
            for (int e = tid; e < (int)(bblock / 4); e += TC_THREADS) {
                float4 x0, x1, x2;
                split3(src[e], x0, x1, x2);
                reinterpret_cast<float4 *>(B0)[e] = x0;
                reinterpret_cast<float4 *>(B1)[e] = x1;
                reinterpret_cast<float4 *>(B2)[e] = x2;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int kvalid = min(TC_KC, P - kc * TC_KC);
            const int nsteps = (kvalid + 7) / 8;
            const uint32_t a0 = smem_u32(A0), a1 = smem_u32(A1), a2 = smem_u32(A2);
            const uint32_t b0 = smem_u32(B0), b1 = smem_u32(B1), b2 = smem_u32(B2);
            for (int s = 0; s < nsteps; ++s) {
                const uint32_t o = s * 2 * TC_LBO;  // 8 K-elements = two core matrices
                const uint32_t acc = (kc > 0 || s > 0) ? 1u : 0u;
                // smallest terms first
                mma_tf32(tmem, make_desc(a2 + o), make_desc(b0 + o), idesc, acc);
                mma_tf32(tmem, make_desc(a1 + o), make_desc(b1 + o), idesc, 1u);
                mma_tf32(tmem, make_desc(a0 + o), make_desc(b2 + o), idesc, 1u);
                mma_tf32(tmem, make_desc(a1 + o), make_desc(b0 + o), idesc, 1u);
                mma_tf32(tmem, make_desc(a0 + o), make_desc(b1 + o), idesc, 1u);
                mma_tf32(tmem, make_desc(a0 + o), make_desc(b0 + o), idesc, 1u);
            }
            mma_commit(smem_u32(mbar));
        }
        __syncwarp();
        const int timed_out = __syncthreads_or(mbar_wait(smem_u32(mbar), phase) ? 0 : 1);
        if (timed_out) {
            // give the in-flight MMAs one more bounded wait before the tensor memory is freed
            mbar_wait(smem_u32(mbar), phase);
            if (tid == 0) atomicOr(err, 1);
            ok = false;
        }
        phase ^= 1u;
        __syncthreads();
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
        // epilogue: warp w holds TMEM lanes 32w..32w+31 = tile rows; 16 columns per load
        const int row = warp * 32 + lane;
        const bool vrow = row < nrows;
        float *yrow = vrow ? Ypair + ((size_t)(ch.start + row / R) * R + (row % R)) * P : nullptr;
        for (int c0 = 0; c0 < Npad; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (vrow) {
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (c0 + i < P) yrow[c0 + i] = __uint_as_float(v[i]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
}

}  // namespace

bool m2l_tc_supported(int P) { return P % 4 == 0 && P <= 256; }

void build_tc_tables(Context &c) {
    Operators &o = c.ops;
    const int P = o.P;
    if (!m2l_tc_supported(P)) return;
    o.tc_Npad = (P + 15) / 16 * 16;
    o.tc_Kpad = (P + TC_KC - 1) / TC_KC * TC_KC;
    size_t per = (size_t)o.tc_Npad * o.tc_Kpad;
    o.m2l_tc.resize(kNumM2LClasses * per);
    dim3 grid(64, kNumM2LClasses);
    k_build_tc_table<<<grid, 256, 0, c.stream>>>(P, o.tc_Npad, o.tc_Kpad, o.m2l32.p, o.m2l_tc.p);
    BEM_LAUNCH_CHECK();
}

size_t m2l_tc_smem_bytes(int Npad) {
    return (size_t)(3 * TC_M * TC_KC + 3 * Npad * TC_KC) * sizeof(float) + 16 + 1024;
}

template <int R>
void launch_m2l_tc(Context &c, const XChunk *chunks, int64_t nchunks, const float *X, float *Ypair, int *err) {
    const Operators &o = c.ops;
    size_t sm = m2l_tc_smem_bytes(o.tc_Npad);
    static bool attr_set[2] = {false, false};
    if (!attr_set[R == 4]) {  // once, for the largest tile (N_pad = 256)
        BEM_CUDA(cudaFuncSetAttribute(k_m2l_tc<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)m2l_tc_smem_bytes(256)));
        attr_set[R == 4] = true;
    }
    k_m2l_tc<R><<<(unsigned)nchunks, TC_THREADS, sm, c.stream>>>(o.P, o.tc_Npad, o.tc_Kpad, o.m2l_tc.p, chunks,
                                                                 c.tree.m2l_src.p, X, Ypair, err);
    BEM_LAUNCH_CHECK();
}

template void launch_m2l_tc<1>(Context &, const XChunk *, int64_t, const float *, float *, int *);
template void launch_m2l_tc<4>(Context &, const XChunk *, int64_t, const float *, float *, int *);

}  // namespace bem
