// M2L translations on the 5th-generation tensor cores (tcgen05, TMEM accumulators).
//
// For one offset class c and a chunk of (source, target) pairs, the product
//   Y[pair, rhs][n] = sum_k T_c[n][k] X[src, rhs][k]
// is up to four MMA tiles D_t = A_t B^T with M = 128 rows (pair, rhs) each, N = K = K_c, the
// class's truncated size (p_c^2 rounded up to 16; P rounded up without truncation):
// A_t = gathered multipole rows, B = T_c (row n of T_c is K-contiguous, i.e. K-major). The
// tiles share every staged block of T_c, which divides its traffic; a chunk of a class with
// K_c <= 128 has four tiles (TMEM columns 128 apart), the others two (256 apart), so the small
// truncated classes amortise a block's set-up and pipeline fill over twice the rows.
//
// Accuracy: both operands are split into three BF16 pieces, x = x0 + x1 + x2 (x0 = bf16(x),
// x1 = bf16(x - x0), x2 = bf16(x - x0 - x1)), and D accumulates in FP32 the six products with
// i + j <= 2: x0 y0 + (x0 y1 + x1 y0) + (x0 y2 + x1 y1 + x2 y0). The dropped terms and the
// rest of x beyond x2 are ~2^-24 of the product, so the translation is as accurate as an FP32
// product. (Translation sums cancel strongly, so a two-piece split leaves noise near 1e-6 in
// the operator, which a GMRES solve to 1e-6 cannot tolerate.) T_c is split once per operator
// build from its FP64 values; the multipoles are split once per product (k_split_x).
//
// Data movement: K advances 16 at a time (one kind::f16 MMA); each 16-wide K step is one
// pipeline stage holding A (3 pieces x tiles x 128 x 16) and B (3 pieces x N_pad x 16) in
// the canonical K-major layout without swizzle (8-row x 16-byte core matrices, K-adjacent core
// matrices 128 B apart, 8-row groups 256 B apart). The block is warp-specialised: warps 1-7
// fill the stages with cp.async (16-byte copies; rows past the chunk read as zeros), three
// stages deep (two on request), and let each stage's "full"
// mbarrier count their copies' arrival (cp.async.mbarrier.arrive.noinc); one thread of warp 0
// waits on "full", issues the stage's MMAs and commits them to the stage's "empty" mbarrier,
// which releases the stage for refilling. No block-wide barrier runs inside the K loop. Every
// wait is bounded: one that runs out raises a shared abort flag that stops the other side at
// its next wait, sets the error flag, and the block waits (bounded) for its MMAs in flight
// before it releases its tensor memory. The same kernel serves the 4-RHS diagonal product
// (R = 4, N_pad up to 256).
#include <cuda_bf16.h>

#include "internal.h"
#include "tcgen05.cuh"

#include <algorithm>
#include <vector>

namespace bem {
namespace {

constexpr int TC_M = 128;        // rows per tile
constexpr int TC_MAXT = 4;       // tiles per block at most (same class, shared B stages)
constexpr int TC_SMALL_K = 128;  // classes truncated to at most this size take four tiles per block
// bytes of one pipeline stage: A (3 pieces x tiles x 128 x 16 BF16) and B (3 pieces x K_c x 16),
// for four tiles with K_c <= 128 or two tiles with K_c <= 256 (the larger of the two)
constexpr size_t TC_STAGE_BYTES = 3 * 4 * TC_M * 16 * 2 + 3 * 128 * 16 * 2;
constexpr int TC_THREADS = 256;  // 8 warps: two warp groups share the loads and the epilogue

// Row-major T_c [P][P] (FP64) -> per class, per 16-wide K step, per piece, an N_pad x 16
// block in the canonical K-major layout, zero-padded (n >= P or k >= P).
__global__ void k_build_tc_table(int P, int Npad, const double *__restrict__ T, __nv_bfloat16 *__restrict__ out) {
    const int cls = blockIdx.y;
    const int nsteps = Npad / TC_K;
    const size_t blk = (size_t)Npad * TC_K;  // one piece of one K step
    const size_t per_cls = blk * 3 * nsteps;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < blk * nsteps;
         e += (size_t)gridDim.x * blockDim.x) {
        const int ks = (int)(e / blk);
        const int rem = (int)(e % blk);
        // inverse of kmajor_off: rem = (n/8)*128 + (kk/8)*64 + (n%8)*8 + kk%8
        const int g = rem >> 7, r2 = rem & 127;
        const int j = r2 >> 6, r3 = r2 & 63;
        const int n = g * 8 + (r3 >> 3), kk = j * 8 + (r3 & 7);
        const int k = ks * TC_K + kk;
        const double v = (n < P && k < P) ? T[((size_t)cls * P + n) * P + k] : 0.0;
        __nv_bfloat16 b0, b1, b2;
        split3_d(v, b0, b1, b2);
        __nv_bfloat16 *o = out + (size_t)cls * per_cls + (size_t)ks * 3 * blk + rem;
        o[0] = b0;
        o[blk] = b1;
        o[2 * blk] = b2;
    }
}

// Multipoles X [rows][P] (FP32) -> three BF16 planes [3][rows][Kp], zero-padded to Kp.
__global__ void k_split_x(int64_t rows, int P, int Kp, const float *__restrict__ X, __nv_bfloat16 *__restrict__ Xs) {
    const int64_t plane = rows * Kp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < plane; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / Kp;
        const int k = (int)(e % Kp);
        const float v = k < P ? X[r * P + k] : 0.f;
        __nv_bfloat16 b0, b1, b2;
        split3_f(v, b0, b1, b2);
        Xs[e] = b0;
        Xs[plane + e] = b1;
        Xs[2 * plane + e] = b2;
    }
}

struct TcLayout {
    size_t stage_bytes, total;
};

// ST pipeline stages and three mbarriers per stage (empty, full, bfull); the epilogue reuses
// the stages for one tile of FP32 rows (at most N_pad floats each)
__host__ __device__ inline TcLayout tc_layout(int Npad, int ST) {
    TcLayout L;
    L.stage_bytes = TC_STAGE_BYTES;
    const size_t epi = (size_t)TC_M * Npad * 4;
    L.total = (ST * L.stage_bytes > epi ? ST * L.stage_bytes : epi) + 3 * ST * 8 + 16 + 1024;
    return L;
}

// tiles per block and TMEM columns per tile for a class truncated to K_c
__host__ __device__ inline int tc_tiles_for(int Kc) { return Kc <= TC_SMALL_K ? TC_MAXT : 2; }

template <int R, int TC_STAGES>
__global__ void __launch_bounds__(TC_THREADS) k_m2l_tc(int P, int Npad, const __nv_bfloat16 *__restrict__ tcB,
                                                       const XChunk *__restrict__ chunks,
                                                       const int32_t *__restrict__ srcs, int64_t xrows,
                                                       const __nv_bfloat16 *__restrict__ Xs, float *__restrict__ Ypair,
                                                       const int32_t *__restrict__ cls_K, int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned base for the operand stages
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const TcLayout Lo = tc_layout(Npad, TC_STAGES);
    const size_t epi_bytes = (size_t)TC_M * Npad * 4;
    uint64_t *empty = reinterpret_cast<uint64_t *>(
        smem + (TC_STAGES * Lo.stage_bytes > epi_bytes ? TC_STAGES * Lo.stage_bytes : epi_bytes));
    uint64_t *full = empty + TC_STAGES;  // NPROD producer arrivals per use (the gathered A rows)
    uint64_t *bfull = full + TC_STAGES;  // one arrival + the bulk copy's bytes (the block of T_c)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bfull + TC_STAGES);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    constexpr int NPROD = TC_THREADS - 32;  // warps 1.. fill the stages, warp 0 issues the MMAs
    __shared__ int s_src[TC_MAXT * TC_M];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // once a block has reported a wait that ran out, the rest skip their work
    if (*reinterpret_cast<volatile int *>(err) != 0) return;
    const XChunk ch = chunks[blockIdx.x];
    const int nrows = ch.count * R;
    const int ntiles = (nrows + TC_M - 1) / TC_M;
    // the class's truncated size (a multiple of 16, <= Npad): K steps and output columns; small
    // classes take four tiles per block (TMEM columns 128 apart), the others two (256 apart)
    const int Kc = cls_K ? cls_K[ch.cls] : Npad;
    const int nsteps = Kc / TC_K;
    const int tcap = tc_tiles_for(Kc);
    const uint32_t colstride = Kc <= TC_SMALL_K ? 128u : 256u;
    for (int r = tid; r < TC_MAXT * TC_M; r += TC_THREADS) s_src[r] = (r < nrows) ? srcs[ch.start + r / R] : -1;
    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[s])), "r"(NPROD));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bfull[s])));
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "n"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = make_idesc(TC_M, Kc);
    const int Kp = Npad;
    const int64_t plane = xrows * Kp;
    const __nv_bfloat16 *Bc = tcB + (size_t)ch.cls * (Npad / TC_K) * 3 * Npad * TC_K;  // the class's full table
    const uint32_t sbase = smem_u32(smem);
    const uint32_t atile = TC_M * TC_K * 2, apiece = (uint32_t)tcap * atile;
    const uint32_t a_bytes = 3 * apiece;
    const uint32_t bpiece = (uint32_t)Kc * TC_K * 2;        // one piece's K_c rows in shared memory
    const size_t bpiece_g = (size_t)Npad * TC_K * 2;        // one piece's block in the table

    // Warp-specialised pipeline. Producers (warps 1..) wait until the MMAs that last read a stage
    // are done (its empty barrier), gather their share of the next K step's A rows into it and let
    // the stage's full barrier count their arrival once those copies have landed
    // (cp.async.mbarrier.arrive.noinc); one producer thread also moves the step's block of T_c
    // (three contiguous pieces) with bulk copies counted on bfull. One thread of warp 0 waits for
    // full and bfull, makes the gathered copies visible to the tensor core (proxy fence), issues
    // the step's MMAs and commits them to empty.
    // No block-wide barrier inside the loop; every wait is bounded and a timeout raises the shared
    // abort flag, which stops the other side at its next wait.
    __shared__ int s_last_ks;
    if (warp == 0) {
        if (lane == 0) {
            int ks = 0;
            for (; ks < nsteps; ++ks) {
                const int st = ks % TC_STAGES;
                const uint32_t ph = (uint32_t)((ks / TC_STAGES) & 1);
                if (!mbar_wait(smem_u32(&full[st]), ph) || !mbar_wait(smem_u32(&bfull[st]), ph) || *abort_flag) {
                    *abort_flag = 1;
                    break;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t sa = sbase + st * (uint32_t)Lo.stage_bytes;
                const uint32_t sb = sa + a_bytes;
                for (int t = 0; t < ntiles; ++t) {
                    const uint32_t d = tmem + (uint32_t)t * colstride;
                    const uint32_t a0 = sa + t * atile;
                    // smallest terms first: (2,0) (1,1) (0,2) (1,0) (0,1) (0,0)
                    mma_bf16(d, make_desc(a0 + 2 * apiece), make_desc(sb), idesc, ks > 0 ? 1u : 0u);
                    mma_bf16(d, make_desc(a0 + apiece), make_desc(sb + bpiece), idesc, 1u);
                    mma_bf16(d, make_desc(a0), make_desc(sb + 2 * bpiece), idesc, 1u);
                    mma_bf16(d, make_desc(a0 + apiece), make_desc(sb), idesc, 1u);
                    mma_bf16(d, make_desc(a0), make_desc(sb + bpiece), idesc, 1u);
                    mma_bf16(d, make_desc(a0), make_desc(sb), idesc, 1u);
                }
                mma_commit(smem_u32(&empty[st]));
            }
            s_last_ks = ks - 1;  // last committed step (-1: none)
        }
        __syncwarp();
    } else {
        const int pt = tid - 32;
        // this thread's A copies, fixed for the block: unit u = (tile row, 8-element half j) of every
        // K step; its three pieces are one plane apart in Xs and one piece block apart in a stage
        constexpr int AU = (TC_MAXT * TC_M * 2 + NPROD - 1) / NPROD;
        const int arows = ntiles * TC_M;
        const __nv_bfloat16 *a_src[AU];
        uint32_t a_dst[AU], a_sz[AU];
#pragma unroll
        for (int i = 0; i < AU; ++i) {
            const int u = pt + i * NPROD;
            const int j = u & 1, row2 = u >> 1;
            const int s = u < 2 * arows ? s_src[row2] : -1;
            a_src[i] = Xs + ((size_t)(s >= 0 ? s : 0) * R + row2 % R) * Kp + j * 8;
            a_dst[i] = (uint32_t)((row2 / TC_M) * atile + kmajor_off(row2 % TC_M, j * 8) * 2);
            a_sz[i] = s >= 0 ? 16u : 0u;  // rows past the chunk: zeros, nothing read
        }
        const bool bulk = pt == 0;
        int issued = -1;  // last K step whose block of T_c this thread requested
        for (int ks = 0; ks < nsteps; ++ks) {
            const int st = ks % TC_STAGES;
            // the stage's previous use (step ks - ST) must be consumed: completion ks / ST - 1
            if (ks >= TC_STAGES &&
                (!mbar_wait(smem_u32(&empty[st]), (uint32_t)((ks / TC_STAGES - 1) & 1)) || *abort_flag)) {
                *abort_flag = 1;
                break;
            }
            const uint32_t sa = sbase + st * (uint32_t)Lo.stage_bytes;
            if (bulk) {
                // B: the first K_c rows of each piece's pre-tiled block (8-row core-matrix groups are
                // contiguous, so that is a prefix of the block)
                const uint32_t bb = smem_u32(&bfull[st]);
                mbar_expect_tx(bb, 3u * bpiece);
                const unsigned char *bsrc = reinterpret_cast<const unsigned char *>(Bc + (size_t)ks * 3 * Npad * TC_K);
                for (int piece = 0; piece < 3; ++piece)
                    bulk_g2s(sa + a_bytes + piece * bpiece, bsrc + (size_t)piece * bpiece_g, bpiece, bb);
                issued = ks;
            }
#pragma unroll
            for (int i = 0; i < AU; ++i) {
                if (pt + i * NPROD < 2 * arows) {
                    const __nv_bfloat16 *src = a_src[i] + ks * TC_K;
                    const uint32_t dst = sa + a_dst[i];
                    cp_async16(dst, src, a_sz[i]);
                    cp_async16(dst + apiece, src + plane, a_sz[i]);
                    cp_async16(dst + 2 * apiece, src + 2 * plane, a_sz[i]);
                }
            }
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&full[st])) : "memory");
        }
        cp_async_wait<0>();  // nothing of this thread in flight past this point
        // the bulk copies of the last steps (those an abort left unconsumed included) land before
        // the block moves on: each stage's latest bfull phase completes when its copy has landed
        for (int ks = issued; ks >= 0 && ks > issued - TC_STAGES; --ks)
            if (!mbar_wait(smem_u32(&bfull[ks % TC_STAGES]), (uint32_t)((ks / TC_STAGES) & 1))) *abort_flag = 1;
    }
    __syncthreads();
    // tcgen05.commit tracks every earlier MMA of the issuing thread: the last commit covers all
    const int lk = s_last_ks;
    const bool done = lk >= 0 && mbar_wait(smem_u32(&empty[lk % TC_STAGES]), (uint32_t)((lk / TC_STAGES) & 1));
    bool ok = !*abort_flag && lk == nsteps - 1 && done;
    if (!ok && tid == 0) atomicOr(err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
        // epilogue, one tile at a time: warp w holds TMEM lanes 32w..32w+31 = tile rows; each
        // thread moves its row into shared memory (row stride P floats: conflict-free 16-byte
        // stores), then the block writes the tile's rows, which are contiguous in Ypair, with
        // coalesced 16-byte stores
        float *stage = reinterpret_cast<float *>(smem);  // the operand stages are free now
        for (int t = 0; t < ntiles; ++t) {
            const int rows_t = min(TC_M, nrows - t * TC_M);
            // a warp reads its own quarter of the TMEM lanes (warp % 4); the two warp groups take
            // the lower and the upper half of the 16-column groups
            const int q4 = warp & 3, half = warp >> 2;
            const int ngroups = Npad / 16, g0 = half ? (ngroups + 1) / 2 : 0, g1 = half ? ngroups : (ngroups + 1) / 2;
            float *srow = stage + (size_t)(q4 * 32 + lane) * P;
            for (int c0 = g0 * 16; c0 < g1 * 16; c0 += 16) {
                if (c0 >= Kc) continue;  // beyond the class's truncation: neither computed nor stored
                uint32_t v[16];
                const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)t * colstride + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int i = 0; i < 16; i += 4)
                    if (c0 + i < P)  // P % 4 == 0: whole 16-byte groups
                        *reinterpret_cast<float4 *>(srow + c0 + i) =
                            make_float4(__uint_as_float(v[i]), __uint_as_float(v[i + 1]), __uint_as_float(v[i + 2]),
                                        __uint_as_float(v[i + 3]));
            }
            __syncthreads();
            float4 *dst = reinterpret_cast<float4 *>(Ypair + ((size_t)ch.start * R + t * TC_M) * P);
            const float4 *src = reinterpret_cast<const float4 *>(stage);
            if (Kc >= P) {
                const int n4 = rows_t * P / 4;
                for (int e = tid; e < n4; e += TC_THREADS) dst[e] = src[e];
            } else {  // the first Kc coefficients of each row; the per-target sums read no more
                const int k4 = Kc / 4, p4 = P / 4;
                for (int e = tid; e < rows_t * k4; e += TC_THREADS) {
                    const int row = e / k4, col = e - row * k4;
                    dst[row * p4 + col] = src[row * p4 + col];
                }
            }
            __syncthreads();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(512));
}

}  // namespace

bool m2l_tc_supported(int P) { return P % 4 == 0 && P <= 256; }

int m2l_tc_pairs_per_chunk(int R, int Kc) { return tc_tiles_for(Kc) * TC_M / R; }

void build_tc_tables(Context &c, Operators &o) {
    const int P = o.P;
    if (!m2l_tc_supported(P)) return;
    o.tc_Npad = (P + 15) / 16 * 16;
    o.tc_Kpad = o.tc_Npad;
    const size_t per = (size_t)3 * o.tc_Npad * o.tc_Kpad;
    o.m2l_tc.resize(kNumM2LClasses * per);
    dim3 grid(64, kNumM2LClasses);
    k_build_tc_table<<<grid, 256, 0, c.stream>>>(P, o.tc_Npad, o.m2l64.p,
                                                 reinterpret_cast<__nv_bfloat16 *>(o.m2l_tc.p));
    BEM_LAUNCH_CHECK();
}

template <int R>
void launch_m2l_tc(Context &c, const Operators &o, const XChunk *chunks, int64_t nchunks, const float *X,
                   int64_t xrows, float *Ypair, int *err, cudaStream_t st) {
    const int Npad = o.tc_Npad;
    // split the multipoles once for all translations of this product
    const size_t nxs = (size_t)3 * xrows * Npad;
    c.xsplit.resize(nxs);
    __nv_bfloat16 *xs = reinterpret_cast<__nv_bfloat16 *>(c.xsplit.p);
    {
        const int64_t plane = xrows * Npad;
        const int nb = (int)std::min<int64_t>(div_up(plane, 256), 152 * 16);
        k_split_x<<<nb, 256, 0, st>>>(xrows, o.P, Npad, X, xs);
        BEM_LAUNCH_CHECK();
    }
    // pipeline depth: the context's choice (parameter or autotuner), else three stages (as many as
    // fit at the four-tile stage size)
    const int stages = c.tuned_stages == 2 ? 2 : 3;
    const size_t sm = tc_layout(Npad, stages).total;
    auto kern = stages == 2 ? k_m2l_tc<R, 2> : k_m2l_tc<R, 3>;
    // set on every launch: the attribute belongs to the current device (~1 us against a ms kernel)
    BEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    kern<<<(unsigned)nchunks, TC_THREADS, sm, st>>>(o.P, Npad, reinterpret_cast<const __nv_bfloat16 *>(o.m2l_tc.p),
                                                   chunks, c.tree.m2l_src.p, xrows, xs, Ypair,
                                                   o.margin >= 0 ? o.cls_K.p : nullptr, err);
    BEM_LAUNCH_CHECK();
}

template void launch_m2l_tc<1>(Context &, const Operators &, const XChunk *, int64_t, const float *, int64_t, float *,
                               int *, cudaStream_t);
template void launch_m2l_tc<4>(Context &, const Operators &, const XChunk *, int64_t, const float *, int64_t, float *,
                               int *, cudaStream_t);

// ------------------------------------------------------------------------------ target-major form
//
// Instead of one output row per translation (summed per target afterwards), a block
// accumulates, for a tile of 256 rows = 256 / R target boxes x R right-hand sides (two M = 128
// tensor-memory accumulators), the translations of a few offset classes: for class c a row's A is
// the multipole of its target's class-c source for its right-hand side (zero rows where a target
// has none), B = T_c, and the MMAs of all the item's classes accumulate into the same columns
// (N = K_c per class), zeroed first. The pipeline is the pair-major kernel's (gathered A rows by
// cp.async, T_c blocks by bulk copies, one MMA thread, bounded waits), but it runs across the
// item's classes without a break. The FP32 accumulation runs from small terms to large: classes
// by truncated size ascending (the far classes, whose translations are the smallest), and within
// a class the K steps from the highest degrees down. A target's items are summed by k_tm_reduce
// in a fixed order with TwoSum compensation, so the FP32 accumulation in tensor memory spans at
// most a few classes (8 for one RHS, 4 for four). Target boxes are grouped by octant (their
// position in the parent), since the 189 classes a box can have depend on it: a tile's classes
// are then about two thirds full. The products use it with one RHS; with four (the diagonal
// product, 64 targets per tile) it was slower than the pair-major kernel.
namespace {

constexpr int TM_ROWS = 2 * TC_M;  // rows per tile: (target, rhs)
constexpr int TM_MAXCLS = 8;       // classes per item at most
constexpr size_t TM_STAGE_BYTES = 3 * TM_ROWS * 16 * 2 + 3 * 256 * 16 * 2;  // A (two tiles) + B (K_c <= 256)

// target boxes: the boxes of levels 2.. with at least one M2L translation, key = octant
__global__ void k_tm_flags(int64_t first, int64_t n, const int32_t *__restrict__ tgt_off, int32_t *__restrict__ flag) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) flag[i] = tgt_off[first + i + 1] > tgt_off[first + i] ? 1 : 0;
}
__global__ void k_tm_emit(int64_t first, int64_t n, const int32_t *__restrict__ flag, const int32_t *__restrict__ ex,
                          const uint32_t *__restrict__ bkey, uint32_t *__restrict__ key, int32_t *__restrict__ box) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && flag[i]) {
        key[ex[i]] = bkey[first + i] & 7u;
        box[ex[i]] = (int32_t)(first + i);
    }
}
__global__ void k_tm_slots(int64_t ntgt, int64_t nslots, const int32_t *__restrict__ sorted,
                           int32_t *__restrict__ tm_box, int32_t *__restrict__ pos) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nslots) return;
    const int32_t b = i < ntgt ? sorted[i] : -1;
    tm_box[i] = b;
    if (b >= 0) pos[b] = (int32_t)i;
}
// every translation (s -> t, class c) fills its (tile, class, slot) entry; TT targets per tile
__global__ void k_tm_fill(int64_t np, int TT, const int32_t *__restrict__ src, const int32_t *__restrict__ tgt,
                          const uint32_t *__restrict__ cls, const int32_t *__restrict__ pos, int32_t *__restrict__ tab) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= np) return;
    const int32_t r = pos[tgt[k]];
    const int64_t tile = r / TT, slot = r % TT;
    tab[(tile * kNumM2LClasses + cls[k]) * TT + slot] = src[k];
}
// per tile, the classes present, in the order `order` (truncated size ascending)
__global__ void __launch_bounds__(512) k_tm_classes(int TT, const int32_t *__restrict__ tab,
                                                    const int32_t *__restrict__ order, int32_t *__restrict__ tcls,
                                                    int32_t *__restrict__ ncls) {
    __shared__ int warp_tot[16];
    const int tile = blockIdx.x, k = threadIdx.x;
    int f = 0;
    if (k < kNumM2LClasses) {
        const int32_t *col = tab + ((int64_t)tile * kNumM2LClasses + order[k]) * TT;
        for (int r = 0; r < TT && !f; ++r) f = col[r] >= 0;
    }
    // block prefix sum of the flags (warp scans, then the warp totals)
    const int lane = k & 31, w = k >> 5;
    int v = f;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) warp_tot[w] = v;
    __syncthreads();
    int before = 0;
    for (int i = 0; i < w; ++i) before += warp_tot[i];
    const int idx = before + v - f;  // exclusive
    if (f) tcls[(int64_t)tile * kNumM2LClasses + idx] = order[k];
    if (k == 511) ncls[tile] = before + v;
}
__global__ void k_tm_item_count(int64_t ntiles, int per, const int32_t *__restrict__ ncls, int32_t *__restrict__ cnt) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < ntiles) cnt[t] = (ncls[t] + per - 1) / per;
}
__global__ void k_tm_item_emit(int64_t ntiles, int per, const int32_t *__restrict__ ncls,
                               const int32_t *__restrict__ off, const int32_t *__restrict__ tcls,
                               const int32_t *__restrict__ cls_K, int Npad, int4 *__restrict__ items) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const int n = ncls[t];
    for (int c0 = 0, i = 0; c0 < n; c0 += per, ++i) {
        const int nc = min(per, n - c0);
        const int last = tcls[t * kNumM2LClasses + c0 + nc - 1];  // the largest truncated size
        items[off[t] + i] = make_int4((int)t, c0, nc, cls_K ? cls_K[last] : Npad);
    }
}

__device__ __forceinline__ void two_sum_add(float &s, float &c, float v) {
    const float t = s + v, bp = t - s;
    c += (s - (t - bp)) + (v - bp);
    s = t;
}

// lc[box][rhs][col] = sum over the tile's items of the partial row (fixed order, compensated)
// (the loads of four items are issued before their sums, which stay in item order; a row's
// coefficients past an item's size read as zero and leave the TwoSum unchanged)
constexpr int TM_MAXITEMS = (kNumM2LClasses + 3) / 4;  // items of one tile at most (4 classes per item)
template <int R>
__global__ void k_tm_reduce(int P, int Npad, const int32_t *__restrict__ tm_box, const int32_t *__restrict__ item_off,
                            const int4 *__restrict__ items, const float *__restrict__ part, float *__restrict__ lc) {
    constexpr int TT = TM_ROWS / R;
    __shared__ int s_kmax[TM_MAXITEMS];
    const int64_t tile = blockIdx.x;
    const int row = blockIdx.y;
    const int32_t box = tm_box[tile * TT + row / R];
    if (box < 0) return;  // uniform in the block
    const int i0 = item_off[tile], i1 = item_off[tile + 1], ni = i1 - i0;
    for (int i = threadIdx.x; i < ni; i += blockDim.x) s_kmax[i] = items[i0 + i].w;
    __syncthreads();
    float *dst = lc + ((int64_t)box * R + row % R) * P;
    const float *src = part + ((int64_t)i0 * TM_ROWS + row) * Npad;
    const int64_t istride = (int64_t)TM_ROWS * Npad;
    for (int col = threadIdx.x; col < P; col += blockDim.x) {
        float s = 0.f, c = 0.f;
        int i = 0;
        for (; i + 4 <= ni; i += 4) {
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = col < s_kmax[i + u] ? src[(i + u) * istride + col] : 0.f;
#pragma unroll
            for (int u = 0; u < 4; ++u) two_sum_add(s, c, v[u]);
        }
        for (; i < ni; ++i)
            if (col < s_kmax[i]) two_sum_add(s, c, src[i * istride + col]);
        dst[col] = s + c;
    }
}

template <int R, int TC_STAGES>
__global__ void __launch_bounds__(TC_THREADS) k_m2l_tm(int P, int Npad, const __nv_bfloat16 *__restrict__ tcB,
                                                       const int4 *__restrict__ items, const int32_t *__restrict__ tab,
                                                       const int32_t *__restrict__ tcls, int64_t xrows,
                                                       const __nv_bfloat16 *__restrict__ Xs, float *__restrict__ part,
                                                       const int32_t *__restrict__ cls_K, int *__restrict__ err) {
    constexpr int TT = TM_ROWS / R;  // target slots per tile
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const size_t stage_bytes = TM_STAGE_BYTES;
    const size_t epi_bytes = (size_t)TC_M * Npad * 4;
    uint64_t *empty = reinterpret_cast<uint64_t *>(
        smem + (TC_STAGES * stage_bytes > epi_bytes ? TC_STAGES * stage_bytes : epi_bytes));
    uint64_t *full = empty + TC_STAGES;
    uint64_t *bfull = full + TC_STAGES;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bfull + TC_STAGES);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    constexpr int NPROD = TC_THREADS - 32;
    __shared__ int s_src[TM_MAXCLS * TT];
    __shared__ int s_cls[TM_MAXCLS], s_K[TM_MAXCLS];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (*reinterpret_cast<volatile int *>(err) != 0) return;
    const int4 it = items[blockIdx.x];
    const int64_t tile = it.x;
    const int nc = it.z, kmax = it.w;
    if (tid < nc) {
        const int cl = tcls[tile * kNumM2LClasses + it.y + tid];
        s_cls[tid] = cl;
        s_K[tid] = cls_K ? cls_K[cl] : Npad;
    }
    __syncthreads();
    for (int e = tid; e < nc * TT; e += TC_THREADS) {
        const int j = e / TT, r = e % TT;
        s_src[e] = tab[(tile * kNumM2LClasses + s_cls[j]) * TT + r];
    }
    int nsteps = 0;
    for (int j = 0; j < nc; ++j) nsteps += s_K[j] / TC_K;
    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[s])), "r"(NPROD));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bfull[s])));
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "n"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    {
        // zero the accumulators' first kmax columns: warp w writes its lane quarter (w % 4) of
        // tile w / 4; every MMA then accumulates
        const uint32_t zr = 0u;
        const uint32_t tb = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(warp >> 2) * 256u;
        for (int c0 = 0; c0 < kmax; c0 += 16)
            asm volatile(
                "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(
                    tb + (uint32_t)c0),
                "r"(zr)
                : "memory");
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    const int Kp = Npad;
    const int64_t plane = xrows * Kp;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t atile = TC_M * TC_K * 2, apiece = 2 * atile;
    const uint32_t a_bytes = 3 * apiece;
    const size_t bpiece_g = (size_t)Npad * TC_K * 2;
    const size_t cls_stride = (size_t)(Npad / TC_K) * 3 * Npad * TC_K;  // elements of one class's table

    __shared__ int s_last_ks;
    if (warp == 0) {
        if (lane == 0) {
            int ks = 0;
            bool stop = false;
            for (int j = 0; j < nc && !stop; ++j) {
                const int Kj = s_K[j];
                const uint32_t idesc = make_idesc(TC_M, Kj);
                const uint32_t bpiece = (uint32_t)Kj * TC_K * 2;
                for (int s = 0; s < Kj / TC_K; ++s, ++ks) {  // K steps from the highest degrees down
                    const int st = ks % TC_STAGES;
                    const uint32_t ph = (uint32_t)((ks / TC_STAGES) & 1);
                    if (!mbar_wait(smem_u32(&full[st]), ph) || !mbar_wait(smem_u32(&bfull[st]), ph) || *abort_flag) {
                        *abort_flag = 1;
                        stop = true;
                        break;
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t sa = sbase + st * (uint32_t)stage_bytes;
                    const uint32_t sb = sa + a_bytes;
                    for (int t = 0; t < 2; ++t) {
                        const uint32_t d = tmem + (uint32_t)t * 256u;
                        const uint32_t a0 = sa + t * atile;
                        mma_bf16(d, make_desc(a0 + 2 * apiece), make_desc(sb), idesc, 1u);
                        mma_bf16(d, make_desc(a0 + apiece), make_desc(sb + bpiece), idesc, 1u);
                        mma_bf16(d, make_desc(a0), make_desc(sb + 2 * bpiece), idesc, 1u);
                        mma_bf16(d, make_desc(a0 + apiece), make_desc(sb), idesc, 1u);
                        mma_bf16(d, make_desc(a0), make_desc(sb + bpiece), idesc, 1u);
                        mma_bf16(d, make_desc(a0), make_desc(sb), idesc, 1u);
                    }
                    mma_commit(smem_u32(&empty[st]));
                }
            }
            s_last_ks = ks - 1;
        }
        __syncwarp();
    } else {
        const int pt = tid - 32;
        constexpr int AU = (TM_ROWS * 2 + NPROD - 1) / NPROD;
        uint32_t a_dst[AU];
#pragma unroll
        for (int i = 0; i < AU; ++i) {
            const int u = pt + i * NPROD;
            const int row2 = u >> 1, jh = u & 1;
            a_dst[i] = (uint32_t)((row2 / TC_M) * atile + kmajor_off(row2 % TC_M, jh * 8) * 2);
        }
        const bool bulk = pt == 0;
        int issued = -1, ks = 0;
        bool stop = false;
        for (int j = 0; j < nc && !stop; ++j) {
            const int Kj = s_K[j];
            const uint32_t bpiece = (uint32_t)Kj * TC_K * 2;
            const __nv_bfloat16 *Bc = tcB + (size_t)s_cls[j] * cls_stride;
            const __nv_bfloat16 *a_src[AU];
            uint32_t a_sz[AU];
#pragma unroll
            for (int i = 0; i < AU; ++i) {
                const int u = pt + i * NPROD;
                const int row2 = u >> 1;  // (target slot, rhs) = (row2 / R, row2 % R)
                const int sidx = u < 2 * TM_ROWS ? s_src[j * TT + row2 / R] : -1;
                a_src[i] = Xs + ((size_t)(sidx >= 0 ? sidx : 0) * R + row2 % R) * Kp + (u & 1) * 8;
                a_sz[i] = sidx >= 0 ? 16u : 0u;  // a target without this class: a zero row
            }
            for (int s = 0; s < Kj / TC_K; ++s, ++ks) {
                const int st = ks % TC_STAGES;
                if (ks >= TC_STAGES &&
                    (!mbar_wait(smem_u32(&empty[st]), (uint32_t)((ks / TC_STAGES - 1) & 1)) || *abort_flag)) {
                    *abort_flag = 1;
                    stop = true;
                    break;
                }
                const uint32_t sa = sbase + st * (uint32_t)stage_bytes;
                const int kstep = Kj / TC_K - 1 - s;  // highest degrees first
                if (bulk) {
                    const uint32_t bb = smem_u32(&bfull[st]);
                    mbar_expect_tx(bb, 3u * bpiece);
                    const unsigned char *bsrc =
                        reinterpret_cast<const unsigned char *>(Bc + (size_t)kstep * 3 * Npad * TC_K);
                    for (int piece = 0; piece < 3; ++piece)
                        bulk_g2s(sa + a_bytes + piece * bpiece, bsrc + (size_t)piece * bpiece_g, bpiece, bb);
                    issued = ks;
                }
#pragma unroll
                for (int i = 0; i < AU; ++i) {
                    if (pt + i * NPROD < 2 * TM_ROWS) {
                        const __nv_bfloat16 *src = a_src[i] + kstep * TC_K;
                        const uint32_t dst = sa + a_dst[i];
                        cp_async16(dst, src, a_sz[i]);
                        cp_async16(dst + apiece, src + plane, a_sz[i]);
                        cp_async16(dst + 2 * apiece, src + 2 * plane, a_sz[i]);
                    }
                }
                asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&full[st])) : "memory");
            }
        }
        cp_async_wait<0>();
        for (int k2 = issued; k2 >= 0 && k2 > issued - TC_STAGES; --k2)
            if (!mbar_wait(smem_u32(&bfull[k2 % TC_STAGES]), (uint32_t)((k2 / TC_STAGES) & 1))) *abort_flag = 1;
    }
    __syncthreads();
    const int lk = s_last_ks;
    const bool done = lk >= 0 && mbar_wait(smem_u32(&empty[lk % TC_STAGES]), (uint32_t)((lk / TC_STAGES) & 1));
    bool ok = !*abort_flag && lk == nsteps - 1 && done;
    if (!ok && tid == 0) atomicOr(err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
        // epilogue, one tile at a time, as in k_m2l_tc: TMEM -> shared memory -> coalesced rows of
        // the item's partial (the first kmax coefficients; the rest of the row is never read)
        float *stage = reinterpret_cast<float *>(smem);
        float *dst_item = part + (size_t)blockIdx.x * TM_ROWS * Npad;
        for (int t = 0; t < 2; ++t) {
            const int q4 = warp & 3, half = warp >> 2;
            const int ngroups = kmax / 16, g0 = half ? (ngroups + 1) / 2 : 0, g1 = half ? ngroups : (ngroups + 1) / 2;
            float *srow = stage + (size_t)(q4 * 32 + lane) * Npad;
            for (int c0 = g0 * 16; c0 < g1 * 16; c0 += 16) {
                uint32_t v[16];
                const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)t * 256u + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int i = 0; i < 16; i += 4)
                    *reinterpret_cast<float4 *>(srow + c0 + i) =
                        make_float4(__uint_as_float(v[i]), __uint_as_float(v[i + 1]), __uint_as_float(v[i + 2]),
                                    __uint_as_float(v[i + 3]));
            }
            __syncthreads();
            const int k4 = kmax / 4, n4 = Npad / 4;
            float4 *dst = reinterpret_cast<float4 *>(dst_item + (size_t)t * TC_M * Npad);
            const float4 *src = reinterpret_cast<const float4 *>(stage);
            for (int e = tid; e < TC_M * k4; e += TC_THREADS) {
                const int row = e / k4, col = e - row * k4;
                dst[row * n4 + col] = src[row * n4 + col];
            }
            __syncthreads();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(512));
}

}  // namespace

// classes per item: 8 for one RHS; 4 for four (the diagonal product's identities cancel O(1)
// sums down to O(h), which magnifies the rounding of the FP32 accumulation)
template <int R>
static void build_tm_tables(Context &c, const Operators &o, cudaStream_t st) {
    Context::TmState &S = c.tm[R == 1 ? 0 : 1];
    constexpr int TT = TM_ROWS / R;
    const int per = R == 1 ? 8 : 4;
    Tree &t = c.tree;
    const int tb = 256;
    const int64_t first = t.base[2], n = (int64_t)t.nbox - first;
    if (n <= 0 || t.n_m2l == 0) {  // no translations: nothing to launch
        S.ntiles = S.nitems = 0;
        S.ok = true;
        S.ops = &o;
        return;
    }
    DevBuf<int32_t> &flag = S.s_i32[0], &ex = S.s_i32[1], &tot = S.s_i32[2];
    flag.resize(std::max<int64_t>(n, 1));
    ex.resize(std::max<int64_t>(n, 1));
    tot.resize(1);
    k_tm_flags<<<div_up(n, tb), tb, 0, st>>>(first, n, t.m2l_tgt_off.p, flag.p);
    BEM_LAUNCH_CHECK();
    exclusive_scan_i32(flag.p, ex.p, n, tot.p, st);
    int32_t ntgt = 0;
    BEM_CUDA(cudaMemcpyAsync(&ntgt, tot.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    BEM_CUDA(cudaStreamSynchronize(st));
    DevBuf<uint32_t> &key = S.s_u32[0], &ktmp = S.s_u32[1];
    DevBuf<int32_t> &box = S.s_i32[3], &btmp = S.s_i32[4], &pos = S.s_i32[5];
    key.resize(std::max(ntgt, 1));
    ktmp.resize(std::max(ntgt, 1));
    box.resize(std::max(ntgt, 1));
    btmp.resize(std::max(ntgt, 1));
    pos.resize(t.nbox);
    k_tm_emit<<<div_up(n, tb), tb, 0, st>>>(first, n, flag.p, ex.p, t.bkey.p, key.p, box.p);
    BEM_LAUNCH_CHECK();
    if (ntgt > 0) radix_sort_u32(key.p, box.p, ntgt, 3, ktmp.p, btmp.p, st);  // stable: box order within an octant
    const int64_t ntiles = div_up((int64_t)ntgt, TT);
    S.ntiles = ntiles;
    S.box.resize(std::max<int64_t>(ntiles * TT, 1));
    k_tm_slots<<<div_up(ntiles * TT, tb), tb, 0, st>>>(ntgt, ntiles * TT, box.p, S.box.p, pos.p);
    BEM_LAUNCH_CHECK();
    const size_t ntab = (size_t)ntiles * kNumM2LClasses * TT;
    S.src.resize(std::max<size_t>(ntab, 1));
    BEM_CUDA(cudaMemsetAsync(S.src.p, 0xff, std::max<size_t>(ntab, 1) * sizeof(int32_t), st));
    k_tm_fill<<<div_up(t.n_m2l, tb), tb, 0, st>>>(t.n_m2l, TT, t.m2l_src.p, t.m2l_tgt.p, t.m2l_cls.p, pos.p, S.src.p);
    BEM_LAUNCH_CHECK();
    // class order: truncated size ascending, ties by class index
    const int P16 = o.tc_Npad;
    std::vector<int32_t> order(kNumM2LClasses);
    for (int k = 0; k < kNumM2LClasses; ++k) order[k] = k;
    auto Kof = [&](int k) { return o.margin >= 0 ? o.cls_Kh[k] : P16; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return Kof(a) < Kof(b); });
    DevBuf<int32_t> &ncls = S.s_i32[6], &icnt = S.s_i32[7];
    DevBuf<int32_t> dorder;
    dorder.resize(kNumM2LClasses);
    ncls.resize(std::max<int64_t>(ntiles, 1));
    icnt.resize(ntiles + 1);
    BEM_CUDA(cudaMemcpyAsync(dorder.p, order.data(), kNumM2LClasses * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    S.cls.resize(std::max<int64_t>(ntiles * kNumM2LClasses, 1));
    S.item_off.resize(ntiles + 1);
    k_tm_classes<<<(unsigned)ntiles, 512, 0, st>>>(TT, S.src.p, dorder.p, S.cls.p, ncls.p);
    BEM_LAUNCH_CHECK();
    k_tm_item_count<<<div_up(ntiles, tb), tb, 0, st>>>(ntiles, per, ncls.p, icnt.p);
    BEM_LAUNCH_CHECK();
    exclusive_scan_i32(icnt.p, S.item_off.p, ntiles, tot.p, st);
    BEM_CUDA(cudaMemcpyAsync(S.item_off.p + ntiles, tot.p, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    int32_t nitems = 0;
    BEM_CUDA(cudaMemcpyAsync(&nitems, tot.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    BEM_CUDA(cudaStreamSynchronize(st));
    S.nitems = nitems;
    S.items.resize(std::max(nitems, 1));
    k_tm_item_emit<<<div_up(ntiles, tb), tb, 0, st>>>(ntiles, per, ncls.p, S.item_off.p, S.cls.p,
                                                       o.margin >= 0 ? o.cls_K.p : nullptr, P16, S.items.p);
    BEM_LAUNCH_CHECK();
    S.part.resize(std::max<size_t>((size_t)nitems * TM_ROWS * P16, 1));
    BEM_CUDA(cudaStreamSynchronize(st));  // dorder is freed on return
    S.ok = true;
    S.ops = &o;
}

template <int R>
void launch_m2l_tm(Context &c, const Operators &o, const float *X, int64_t xrows, int *err, cudaStream_t st) {
    Context::TmState &S = c.tm[R == 1 ? 0 : 1];
    if (!S.ok || S.ops != &o) build_tm_tables<R>(c, o, st);
    const int Npad = o.tc_Npad;
    const size_t nxs = (size_t)3 * xrows * Npad;
    c.xsplit.resize(nxs);
    __nv_bfloat16 *xs = reinterpret_cast<__nv_bfloat16 *>(c.xsplit.p);
    {
        const int64_t plane = xrows * Npad;
        const int nb = (int)std::min<int64_t>(div_up(plane, 256), 152 * 16);
        k_split_x<<<nb, 256, 0, st>>>(xrows, o.P, Npad, X, xs);
        BEM_LAUNCH_CHECK();
    }
    if (S.nitems == 0) return;
    const int stages = 3;
    const size_t epi = (size_t)TC_M * Npad * 4;
    const size_t sm = (stages * TM_STAGE_BYTES > epi ? stages * TM_STAGE_BYTES : epi) + 3 * stages * 8 + 16 + 1024;
    BEM_CUDA(cudaFuncSetAttribute(k_m2l_tm<R, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_m2l_tm<R, 3><<<(unsigned)S.nitems, TC_THREADS, sm, st>>>(
        o.P, Npad, reinterpret_cast<const __nv_bfloat16 *>(o.m2l_tc.p), S.items.p, S.src.p, S.cls.p, xrows, xs, S.part.p,
        o.margin >= 0 ? o.cls_K.p : nullptr, err);
    BEM_LAUNCH_CHECK();
}

template <int R>
void launch_m2l_tm_reduce(Context &c, const Operators &o, float *lc, cudaStream_t st) {
    Context::TmState &S = c.tm[R == 1 ? 0 : 1];
    if (S.nitems == 0) return;
    dim3 grid((unsigned)S.ntiles, TM_ROWS);
    k_tm_reduce<R><<<grid, 128, 0, st>>>(o.P, o.tc_Npad, S.box.p, S.item_off.p, S.items.p, S.part.p, lc);
    BEM_LAUNCH_CHECK();
}

template void launch_m2l_tm<1>(Context &, const Operators &, const float *, int64_t, int *, cudaStream_t);
template void launch_m2l_tm_reduce<1>(Context &, const Operators &, float *, cudaStream_t);

}  // namespace bem
