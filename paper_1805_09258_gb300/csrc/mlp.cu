// mlp.cu -- learned radius predictor (not in the paper): coarse features, a
// 256-64-64-1 GELU MLP on the 5th-generation tensor cores, its training step, AdamW.
//
// Features (k_coarse_features): for the coarse stratified ray set of a position, the
// log distance to the first hit (or cube exit) and the to-light transmittance times
// visibility at that point -- 2 N values per record.
//
// Network: z1 = W1 x + b1, h1 = gelu(z1), z2 = W2 h1 + b2, h2 = gelu(z2), y = w3 . h2 + b3
// (y = predicted log radius), loss = mean (y - t)^2.  BF16 operands (x, W1, W2, w3, h1;
// dz2 and dz1 where they are GEMM operands), FP32 accumulation in tensor memory.
//
// Tensor-core mapping, one tile of 128 records per step of a block of 128 threads
// (thread t owns record row t, i.e. tensor-memory lane t):
//   forward   D1[128x64] = X[128x256] W1^T,    D2[128x64] = H1[128x64] W2^T
//   backward  D3[128x64] = dZ2[128x64] W2        (dh1)
//             E0,E1[128x64] = X^T[256x128] dZ1  (dW1^T, two 128-row tiles, K = records)
//             E2[128x64] = [H1^T; 0][128x128] dZ2 (dW2^T in rows 0..63, K = records)
// Operands live in shared memory in the 128-byte-swizzled K-major layout (8 rows x 128 B
// atoms, 16-byte chunk c of row r stored at chunk c ^ (r & 7)); tcgen05.mma is issued by
// one thread and signals an mbarrier through tcgen05.commit; results are read back with
// tcgen05.ld (32 lanes x 32 bit per warp).  The weight-gradient accumulators E0..E2 stay
// in tensor memory across a block's tiles and are added to global memory once.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "vrc_internal.cuh"

#define MLP_IN 256
#define MLP_H 64
#define MLP_NPARAM (MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1)
#define OFF_W1 0
#define OFF_B1 (MLP_H * MLP_IN)
#define OFF_W2 (OFF_B1 + MLP_H)
#define OFF_B2 (OFF_W2 + MLP_H * MLP_H)
#define OFF_W3 (OFF_B2 + MLP_H)
#define OFF_B3 (OFF_W3 + MLP_H)

struct vrc_mlp {
    float* params;      // fp32 master parameters [MLP_NPARAM]
    float* grad;        // [MLP_NPARAM]
    float* m;           // AdamW moments
    float* v;
    float* loss;        // [1]: sum of squared residuals of the last gradient call
    float* partial;     // [blocks][MLP_NPARAM + 1]: per-block gradients and loss
    int partial_blocks;
    int* err;           // device error flag (bounded waits)
    long long step;
};

namespace {

// ------------------------------------------------------------------ coarse features
__device__ __forceinline__ void st_feat(float* f, size_t i, float v) { f[i] = v; }
__device__ __forceinline__ void st_feat(__nv_bfloat16* f, size_t i, float v) { f[i] = __float2bfloat16_rn(v); }

// T = float, or __nv_bfloat16 (rounded to nearest even: the value the forward pass would
// round the float feature to when staging it as a tensor-core operand)
template <typename T>
__global__ void k_coarse_features(DevScene sc, const float* pos, int n, int nb, int ns, uint64_t seed,
                                  long long rec_base, T* feat) {
    const int N = nb * ns;
    for (long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x; item < (long long)n * N;
         item += (long long)gridDim.x * blockDim.x) {
        int rec = (int)(item / N), v = (int)(item - (long long)rec * N);
        float3 x = f3(pos[3 * rec], pos[3 * rec + 1], pos[3 * rec + 2]);
        float3 d = ray_direction_dev(seed, rec_base + rec, v, nb, ns);
        float th;
        int prim = bvh_trace<false>(sc, x, d, VRC_TMIN, 3.0e38f, &th);
        float t = prim >= 0 ? th : cube_exit_dev(x, d);
        float3 y = x + d * t, o = y;
        if (prim >= 0) {
            float4 n4 = __ldg(&sc.prim[3 * prim]);
            float3 nn = f3(n4.x, n4.y, n4.z);
            if (dot3(nn, d) > 0.f) nn = nn * -1.0f;
            o = y + nn * 1e-5f;
        }
        float tv = 0.f;
        for (int l = 0; l < sc.n_lights; ++l) {
            float3 lo = sc.lpos[l] - o;
            float dl = sqrtf(dot3(lo, lo));
            if (shadow_occluded(sc, l, o, lo * (1.0f / dl), dl)) continue;
            float3 ly = sc.lpos[l] - y;
            tv += __expf(-sc.sigma_t * sqrtf(dot3(ly, ly)));
        }
        st_feat(feat, (size_t)rec * 2 * N + v, __logf(t));
        st_feat(feat, (size_t)rec * 2 * N + N + v, tv);
    }
}

// ------------------------------------------------------------------ tcgen05 helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: 128-byte swizzle, K-major, 8-row atoms 1024 B apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);       // start address >> 4, bits [0,14)
    d |= (uint64_t)1 << 16;                         // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;               // stride byte offset: next 8-row atom
    d |= (uint64_t)1 << 46;                         // descriptor version
    d |= (uint64_t)2 << 61;                         // layout: 128-byte swizzle
    return d;
}

// instruction descriptor: kind::f16 with BF16 A and B, FP32 D, both K-major, M = 128
__device__ __forceinline__ uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, int accum) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");   // visible to the tensor-core arrive
}

// bounded wait for the given phase parity; returns false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (long long it = 0; it < (1ll << 26); ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&r)[16]) {
    uint32_t u[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
          "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) r[i] = __uint_as_float(u[i]);
}

// byte offset of element (row, k) of a K-major operand with `rows` rows, in 64-wide K blocks
__device__ __forceinline__ uint32_t sw_off(int row, int k, int rows) {
    int kb = k >> 6, kk = k & 63;
    int chunk = kk >> 3;
    return (uint32_t)(kb * rows * 128 + row * 128 + ((chunk ^ (row & 7)) << 4) + ((kk & 7) << 1));
}

__device__ __forceinline__ unsigned short bf16_bits(float f) {
    __nv_bfloat16 b = __float2bfloat16_rn(f);
    return *reinterpret_cast<unsigned short*>(&b);
}
__device__ __forceinline__ float bf16_round(float f) { return __bfloat162float(__float2bfloat16_rn(f)); }

__device__ __forceinline__ void st_bf16(unsigned char* base, uint32_t off, float f) {
    *reinterpret_cast<unsigned short*>(base + off) = bf16_bits(f);
}

// 8 consecutive K elements of one row (a 16-byte chunk), k0 a multiple of 8
__device__ __forceinline__ void st_chunk(unsigned char* base, int row, int k0, int rows, const float* v8) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) w[i] = (uint32_t)bf16_bits(v8[2 * i]) | ((uint32_t)bf16_bits(v8[2 * i + 1]) << 16);
    *reinterpret_cast<uint4*>(base + sw_off(row, k0, rows)) = make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * __expf(-0.5f * z * z) * 0.39894228040143268f;
}

// stage a [rows x K] fp32 row-major matrix (ld floats per row) as BF16 K-major swizzled
__device__ void stage_rows(unsigned char* base, const float* src, int rows, int valid_rows, int K, int ld) {
    int chunks = rows * (K / 8);
    for (int q = threadIdx.x; q < chunks; q += blockDim.x) {
        int row = q / (K / 8), k0 = (q - row * (K / 8)) * 8;
        float v[8];
        if (row < valid_rows) {
            const float4* s4 = reinterpret_cast<const float4*>(src + (size_t)row * ld + k0);
            float4 a = s4[0], b = s4[1];
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = 0.f;
        }
        st_chunk(base, row, k0, rows, v);
    }
}

// The same for a [rows x K] tile streamed from HBM: each thread issues the loads of 8 chunks
// before converting any of them, so 8x more bytes are in flight per thread.
__device__ void stage_rows_stream(unsigned char* base, const float* src, int rows, int valid_rows, int K, int ld) {
    const int cpr = K / 8, chunks = rows * cpr;
    for (int q0 = threadIdx.x; q0 < chunks; q0 += 8 * blockDim.x) {
        float4 a[8], b[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int q = q0 + u * blockDim.x;
            const int row = q / cpr, k0 = (q - row * cpr) * 8;
            if (q < chunks && row < valid_rows) {
                const float4* s4 = reinterpret_cast<const float4*>(src + (size_t)row * ld + k0);
                a[u] = __ldcs(s4);
                b[u] = __ldcs(s4 + 1);
            } else {
                a[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                b[u] = a[u];
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int q = q0 + u * blockDim.x;
            if (q >= chunks) break;
            const int row = q / cpr, k0 = (q - row * cpr) * 8;
            const float v[8] = {a[u].x, a[u].y, a[u].z, a[u].w, b[u].x, b[u].y, b[u].z, b[u].w};
            st_chunk(base, row, k0, rows, v);
        }
    }
}

// sum of v over the block's 128 threads, in a fixed order (warp butterfly, then warps 0..3)
__device__ __forceinline__ float block_sum_fixed(float v, float* scratch4) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncwarp();
    if ((threadIdx.x & 31) == 0) scratch4[threadIdx.x >> 5] = v;
    __syncthreads();
    float r = ((scratch4[0] + scratch4[1]) + scratch4[2]) + scratch4[3];
    __syncthreads();
    return r;
}

struct MlpSmem {
    // byte offsets inside the 1024-aligned dynamic shared memory
    static constexpr uint32_t X = 0;                       // 128 x 256 (64 KB); training: reused for X^T
    static constexpr uint32_t W1 = X + 65536;              // 64 x 256 (32 KB)
    static constexpr uint32_t W2 = W1 + 32768;             // 64 x 64 (8 KB)
    static constexpr uint32_t W2T = W2 + 8192;             // 64 x 64 (8 KB)
    static constexpr uint32_t H1 = W2T + 8192;             // 128 x 64 (16 KB)
    static constexpr uint32_t H1T = H1 + 16384;            // 128 x 128 (32 KB): rows 0..63 = h1^T, rest 0
    static constexpr uint32_t DZ2 = H1T + 32768;           // 128 x 64 (16 KB)
    static constexpr uint32_t DZ2T = DZ2 + 16384;          // 64 x 128 (16 KB)
    static constexpr uint32_t DZ1T = DZ2T + 16384;         // 64 x 128 (16 KB)
    static constexpr uint32_t END = DZ1T + 16384;          // 212,992
    // forward kernel: X, W1, W2; its H1 reuses X once the first product has read it, so two
    // blocks fit an SM and one block's loads overlap the other's tensor-core work
    static constexpr uint32_t FWD_H1 = X;
    static constexpr uint32_t FWD_END = W2 + 8192;         // 106,496
};

constexpr int TMEM_D1 = 0, TMEM_D2 = 64, TMEM_D3 = 128, TMEM_E0 = 192, TMEM_E1 = 256, TMEM_E2 = 320;

__device__ __forceinline__ void tmem_alloc(uint32_t* holder, int ncols) {
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(holder)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
}
__device__ __forceinline__ void tmem_free(uint32_t base, int ncols) {
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(ncols));
}

// D[128 x n] (+)= A[128 x K] B[n x K]^T with both operands K-major swizzled in smem
__device__ __forceinline__ void mma_tile(uint32_t tmem_d, uint32_t a_base, int a_rows, uint32_t b_base, int b_rows,
                                        int K, int n, int accum_first) {
    uint32_t idesc = idesc_bf16(n);
    for (int kk = 0; kk < K / 16; ++kk) {
        uint32_t koff = (uint32_t)((kk & 3) * 32);           // 16 BF16 = 32 B inside the 128 B swizzle row
        uint64_t a = sw128_desc(a_base + (uint32_t)((kk >> 2) * a_rows * 128) + koff);
        uint64_t b = sw128_desc(b_base + (uint32_t)((kk >> 2) * b_rows * 128) + koff);
        mma_bf16(tmem_d, a, b, idesc, (kk > 0 || accum_first) ? 1 : 0);
    }
}

// ------------------------------------------------------------------ forward (inference)
__global__ void __launch_bounds__(128, 2) k_mlp_forward(const float* __restrict__ prm, const float* __restrict__ X,
                                                        int n, float* __restrict__ y, int* err) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_holder;
    __shared__ float b1s[MLP_H], b2s[MLP_H], w3s[MLP_H];
    const int t = threadIdx.x, warp = t >> 5;
    const uint32_t sbase = smem_addr(sm);
    if (t == 0) mbar_init(smem_addr(&mbar));
    tmem_alloc(&tmem_holder, 128);
    stage_rows(sm + MlpSmem::W1, prm + OFF_W1, MLP_H, MLP_H, MLP_IN, MLP_IN);
    stage_rows(sm + MlpSmem::W2, prm + OFF_W2, MLP_H, MLP_H, MLP_H, MLP_H);
    if (t < MLP_H) {
        b1s[t] = prm[OFF_B1 + t];
        b2s[t] = prm[OFF_B2 + t];
        w3s[t] = bf16_round(prm[OFF_W3 + t]);
    }
    const float b3 = prm[OFF_B3];
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_holder;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    uint32_t phase = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile * 128 < n && ok; tile += gridDim.x) {
        const int r0 = tile * 128;
        const int valid = min(128, n - r0);
        stage_rows_stream(sm + MlpSmem::X, X + (size_t)r0 * MLP_IN, 128, valid, MLP_IN, MLP_IN);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (t == 0) {
            tc_fence_after();
            mma_tile(tmem + TMEM_D1, sbase + MlpSmem::X, 128, sbase + MlpSmem::W1, MLP_H, MLP_IN, MLP_H, 0);
            mma_commit(smem_addr(&mbar));
        }
        ok = mbar_wait(smem_addr(&mbar), phase);
        phase ^= 1;
        tc_fence_after();
        float h[MLP_H];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float r[16];
            tmem_ld16(tmem + lane_off + TMEM_D1 + 16 * c, r);
#pragma unroll
            for (int i = 0; i < 16; ++i) h[16 * c + i] = gelu(r[i] + b1s[16 * c + i]);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) st_chunk(sm + MlpSmem::FWD_H1, t, 8 * c, 128, h + 8 * c);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (t == 0) {
            tc_fence_after();
            mma_tile(tmem + TMEM_D2, sbase + MlpSmem::FWD_H1, 128, sbase + MlpSmem::W2, MLP_H, MLP_H, MLP_H, 0);
            mma_commit(smem_addr(&mbar));
        }
        ok = ok && mbar_wait(smem_addr(&mbar), phase);
        phase ^= 1;
        tc_fence_after();
        float acc = b3;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float r[16];
            tmem_ld16(tmem + lane_off + TMEM_D2 + 16 * c, r);
#pragma unroll
            for (int i = 0; i < 16; ++i) acc = fmaf(w3s[16 * c + i], gelu(r[i] + b2s[16 * c + i]), acc);
        }
        if (t < valid) y[r0 + t] = acc;
        tc_fence_before();
        __syncthreads();
    }
    if (!ok && t == 0) atomicExch(err, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    tmem_free(tmem_holder, 128);
}

// ------------------------------------------------------------------ forward from BF16 features by TMA
// The feature tile X [128 rows x 256] arrives from HBM by four tiled bulk-tensor copies
// (cp.async.bulk.tensor.2d, box 64 features x 128 rows, 128-byte swizzle): each lands as
// one 64-wide K block of the K-major swizzled operand layout above, so the tensor cores
// read it as it is, with no register pass.  Rows past n are filled with zeros by the copy.
// 512 B per record read instead of 1,024 B of FP32; predictions equal k_mlp_forward's on
// the same features rounded to BF16 (its staging rounds them the same way).
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

// One feature buffer per block and two blocks per SM (106 KB of shared memory each): one
// block's copy overlaps the other's tensor-core work and epilogue.  (Two buffers per block
// at one block per SM measured 0.39 ms per 1M rows against 0.22 ms: the per-tile epilogue,
// not the copy, is then the longer part and nothing overlaps it.)
__global__ void __launch_bounds__(128, 2) k_mlp_forward_tma(const __grid_constant__ CUtensorMap tm_x,
                                                            const float* __restrict__ prm, int n,
                                                            float* __restrict__ y, int* err) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t mbar, mbar_x;
    __shared__ uint32_t tmem_holder;
    __shared__ float b1s[MLP_H], b2s[MLP_H], w3s[MLP_H];
    const int t = threadIdx.x, warp = t >> 5;
    const uint32_t sbase = smem_addr(sm);
    if (t == 0) {
        mbar_init(smem_addr(&mbar));
        mbar_init(smem_addr(&mbar_x));
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tm_x)) : "memory");
    }
    tmem_alloc(&tmem_holder, 128);
    stage_rows(sm + MlpSmem::W1, prm + OFF_W1, MLP_H, MLP_H, MLP_IN, MLP_IN);
    stage_rows(sm + MlpSmem::W2, prm + OFF_W2, MLP_H, MLP_H, MLP_H, MLP_H);
    if (t < MLP_H) {
        b1s[t] = prm[OFF_B1 + t];
        b2s[t] = prm[OFF_B2 + t];
        w3s[t] = bf16_round(prm[OFF_W3 + t]);
    }
    const float b3 = prm[OFF_B3];
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_holder;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    uint32_t phase = 0, phase_x = 0;
    bool ok = true, x_pending = false, mma_pending = false;
    for (int tile = blockIdx.x; tile * 128 < n; tile += gridDim.x) {
        const int r0 = tile * 128;
        const int valid = min(128, n - r0);
        if (t == 0) {
            mbar_expect_tx(smem_addr(&mbar_x), 128u * MLP_IN * 2u);
#pragma unroll
            for (int kb = 0; kb < MLP_IN / 64; ++kb)
                tma_load_2d(sbase + MlpSmem::X + (uint32_t)(kb * 128 * 128), &tm_x, kb * 64, r0, smem_addr(&mbar_x));
        }
        x_pending = true;
        ok = mbar_wait(smem_addr(&mbar_x), phase_x);
        if (!ok) break;
        x_pending = false;
        phase_x ^= 1;
        tc_fence_after();
        if (t == 0) {
            mma_tile(tmem + TMEM_D1, sbase + MlpSmem::X, 128, sbase + MlpSmem::W1, MLP_H, MLP_IN, MLP_H, 0);
            mma_commit(smem_addr(&mbar));
        }
        mma_pending = true;
        ok = mbar_wait(smem_addr(&mbar), phase);
        if (!ok) break;
        mma_pending = false;
        phase ^= 1;
        tc_fence_after();
        float h[MLP_H];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float r[16];
            tmem_ld16(tmem + lane_off + TMEM_D1 + 16 * c, r);
#pragma unroll
            for (int i = 0; i < 16; ++i) h[16 * c + i] = gelu(r[i] + b1s[16 * c + i]);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) st_chunk(sm + MlpSmem::FWD_H1, t, 8 * c, 128, h + 8 * c);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (t == 0) {
            tc_fence_after();
            mma_tile(tmem + TMEM_D2, sbase + MlpSmem::FWD_H1, 128, sbase + MlpSmem::W2, MLP_H, MLP_H, MLP_H, 0);
            mma_commit(smem_addr(&mbar));
        }
        mma_pending = true;
        ok = mbar_wait(smem_addr(&mbar), phase);
        if (!ok) break;
        mma_pending = false;
        phase ^= 1;
        tc_fence_after();
        float acc = b3;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float r[16];
            tmem_ld16(tmem + lane_off + TMEM_D2 + 16 * c, r);
#pragma unroll
            for (int i = 0; i < 16; ++i) acc = fmaf(w3s[16 * c + i], gelu(r[i] + b2s[16 * c + i]), acc);
        }
        if (t < valid) y[r0 + t] = acc;
        // the next tile's copy overwrites X (which h1 shares): every thread is past its reads
        tc_fence_before();
        __syncthreads();
    }
    if (!ok) {
        // a wait gave up: flag it, and wait (bounded again) for this block's own copy or
        // tensor-core work still in flight before the shared and tensor memory are released
        if (t == 0) atomicExch(err, 1);
        if (x_pending) mbar_wait(smem_addr(&mbar_x), phase_x);
        if (mma_pending) mbar_wait(smem_addr(&mbar), phase);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    tmem_free(tmem_holder, 128);
}

// ------------------------------------------------------------------ training (gradients)
// part[blockIdx.x][0, MLP_NPARAM) = this block's share of d loss / d params for
// loss = (1 / n) sum (y - t)^2, part[blockIdx.x][MLP_NPARAM] = its sum of squared residuals.
// Every sum runs in a fixed order (tensor-memory accumulation over the block's tiles in
// tile order, fixed warp/lane reduction trees), so gradients are bitwise reproducible.
__global__ void __launch_bounds__(128, 1) k_mlp_grad(const float* __restrict__ prm, const float* __restrict__ X,
                                                     const float* __restrict__ target, int n, float inv_n,
                                                     float* __restrict__ part, float* __restrict__ y_out,
                                                     int* err) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_holder;
    __shared__ float b1s[MLP_H], b2s[MLP_H], w3s[MLP_H];
    __shared__ float gb1[MLP_H], gb2[MLP_H], gw3[MLP_H], gsc[2], red4[4];
    const int t = threadIdx.x, warp = t >> 5;
    const uint32_t sbase = smem_addr(sm);
    if (t == 0) mbar_init(smem_addr(&mbar));
    tmem_alloc(&tmem_holder, 512);
    stage_rows(sm + MlpSmem::W1, prm + OFF_W1, MLP_H, MLP_H, MLP_IN, MLP_IN);
    stage_rows(sm + MlpSmem::W2, prm + OFF_W2, MLP_H, MLP_H, MLP_H, MLP_H);
    // W2^T: row i (input of layer 2), K = o (output): element W2[o][i]
    for (int e = t; e < MLP_H * MLP_H; e += 128) {
        int i = e / MLP_H, o = e - i * MLP_H;
        st_bf16(sm + MlpSmem::W2T, sw_off(i, o, MLP_H), prm[OFF_W2 + o * MLP_H + i]);
    }
    // H1^T rows 64..127 stay zero (padding of the M = 64 product to M = 128)
    for (int e = t; e < 32768 / 16; e += 128) reinterpret_cast<uint4*>(sm + MlpSmem::H1T)[e] = make_uint4(0, 0, 0, 0);
    if (t < MLP_H) {
        b1s[t] = prm[OFF_B1 + t];
        b2s[t] = prm[OFF_B2 + t];
        w3s[t] = bf16_round(prm[OFF_W3 + t]);
        gb1[t] = gb2[t] = gw3[t] = 0.f;
    }
    if (t < 2) gsc[t] = 0.f;
    const float b3 = prm[OFF_B3];
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_holder;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    uint32_t phase = 0;
    bool ok = true;
    int tiles_done = 0;
    for (int tile = blockIdx.x; tile * 128 < n && ok; tile += gridDim.x) {
        const int r0 = tile * 128;
        const int valid = min(128, n - r0);
        const bool live = t < valid;
        // ---- forward layer 1
        stage_rows(sm + MlpSmem::X, X + (size_t)r0 * MLP_IN, 128, valid, MLP_IN, MLP_IN);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (t == 0) {
            tc_fence_after();
            mma_tile(tmem + TMEM_D1, sbase + MlpSmem::X, 128, sbase + MlpSmem::W1, MLP_H, MLP_IN, MLP_H, 0);
            mma_commit(smem_addr(&mbar));
        }
        ok = mbar_wait(smem_addr(&mbar), phase);
        phase ^= 1;
        tc_fence_after();
        float z1[MLP_H];
        {
            float hq[MLP_H];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float r[16];
                tmem_ld16(tmem + lane_off + TMEM_D1 + 16 * c, r);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    z1[16 * c + i] = r[i] + b1s[16 * c + i];
                    hq[16 * c + i] = gelu(z1[16 * c + i]);
                }
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) st_chunk(sm + MlpSmem::H1, t, 8 * c, 128, hq + 8 * c);
            // h1^T for dW2: row = feature, K = record t
#pragma unroll 8
            for (int f = 0; f < MLP_H; ++f) st_bf16(sm + MlpSmem::H1T, sw_off(f, t, 128), hq[f]);
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (t == 0) {
            tc_fence_after();
            mma_tile(tmem + TMEM_D2, sbase + MlpSmem::H1, 128, sbase + MlpSmem::W2, MLP_H, MLP_H, MLP_H, 0);
            mma_commit(smem_addr(&mbar));
        }
        ok = ok && mbar_wait(smem_addr(&mbar), phase);
        phase ^= 1;
        tc_fence_after();
        // ---- forward layer 2, output, loss, dz2
        float z2[MLP_H];
        float yv = b3;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float r[16];
            tmem_ld16(tmem + lane_off + TMEM_D2 + 16 * c, r);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                z2[16 * c + i] = r[i] + b2s[16 * c + i];
                yv = fmaf(w3s[16 * c + i], gelu(z2[16 * c + i]), yv);
            }
        }
        float res = live ? yv - target[r0 + t] : 0.f;
        if (live && y_out) y_out[r0 + t] = yv;
        float dy = 2.0f * res * inv_n;
        {
            float s0 = block_sum_fixed(res * res, red4), s1 = block_sum_fixed(dy, red4);
            if (t == 0) { gsc[0] += s0; gsc[1] += s1; }
        }
        {
            float dz2[MLP_H];
#pragma unroll 4
            for (int j = 0; j < MLP_H; ++j) {
                float hj = gelu(z2[j]);
                dz2[j] = dy * w3s[j] * gelu_d(z2[j]);
                float sw = block_sum_fixed(dy * hj, red4), sb = block_sum_fixed(dz2[j], red4);
                if (t == 0) { gw3[j] += sw; gb2[j] += sb; }
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) st_chunk(sm + MlpSmem::DZ2, t, 8 * c, 128, dz2 + 8 * c);
#pragma unroll 8
            for (int f = 0; f < MLP_H; ++f) st_bf16(sm + MlpSmem::DZ2T, sw_off(f, t, MLP_H), dz2[f]);
        }
        // X^T for dW1 (reuses the X buffer): two 128-row tiles, row = input feature, K = record t
        tc_fence_before();
        __syncthreads();                                   // layer-1 MMA has read X (waited above)
        {
            const float* xr = X + (size_t)(r0 + (live ? t : 0)) * MLP_IN;
            for (int f = 0; f < MLP_IN; ++f) {
                float xv = live ? __ldg(&xr[f]) : 0.f;
                st_bf16(sm + MlpSmem::X + (f >> 7) * 32768, sw_off(f & 127, t, 128), xv);
            }
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (t == 0) {
            tc_fence_after();
            // dh1 = dz2 W2 ; dW2^T += [h1^T; 0] dz2
            mma_tile(tmem + TMEM_D3, sbase + MlpSmem::DZ2, 128, sbase + MlpSmem::W2T, MLP_H, MLP_H, MLP_H, 0);
            mma_tile(tmem + TMEM_E2, sbase + MlpSmem::H1T, 128, sbase + MlpSmem::DZ2T, MLP_H, 128, MLP_H,
                     tiles_done > 0);
            mma_commit(smem_addr(&mbar));
        }
        ok = ok && mbar_wait(smem_addr(&mbar), phase);
        phase ^= 1;
        tc_fence_after();
        {
            float dz1[MLP_H];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float r[16];
                tmem_ld16(tmem + lane_off + TMEM_D3 + 16 * c, r);
#pragma unroll
                for (int i = 0; i < 16; ++i) dz1[16 * c + i] = r[i] * gelu_d(z1[16 * c + i]);
            }
#pragma unroll 4
            for (int j = 0; j < MLP_H; ++j) {
                float sb = block_sum_fixed(dz1[j], red4);
                if (t == 0) gb1[j] += sb;
            }
#pragma unroll 8
            for (int f = 0; f < MLP_H; ++f) st_bf16(sm + MlpSmem::DZ1T, sw_off(f, t, MLP_H), dz1[f]);
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (t == 0) {
            tc_fence_after();
            // dW1^T += X^T dz1 (input features 0..127 and 128..255)
            mma_tile(tmem + TMEM_E0, sbase + MlpSmem::X, 128, sbase + MlpSmem::DZ1T, MLP_H, 128, MLP_H, tiles_done > 0);
            mma_tile(tmem + TMEM_E1, sbase + MlpSmem::X + 32768, 128, sbase + MlpSmem::DZ1T, MLP_H, 128, MLP_H,
                     tiles_done > 0);
            mma_commit(smem_addr(&mbar));
        }
        ok = ok && mbar_wait(smem_addr(&mbar), phase);
        phase ^= 1;
        tc_fence_after();
        ++tiles_done;
    }
    // ---- this block's gradients (a block without tiles writes zeros)
    float* gp = part + (size_t)blockIdx.x * (MLP_NPARAM + 1);
    if (ok) {
#pragma unroll
        for (int half = 0; half < 2; ++half)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float r[16];
                tmem_ld16(tmem + lane_off + (half ? TMEM_E1 : TMEM_E0) + 16 * c, r);
                int f = half * 128 + t;                       // input feature (row of dW1^T)
#pragma unroll
                for (int i = 0; i < 16; ++i) gp[OFF_W1 + (16 * c + i) * MLP_IN + f] = tiles_done ? r[i] : 0.f;
            }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float r[16];
            tmem_ld16(tmem + lane_off + TMEM_E2 + 16 * c, r);  // all lanes load (warp-collective)
            if (t < MLP_H)
#pragma unroll
                for (int i = 0; i < 16; ++i) gp[OFF_W2 + (16 * c + i) * MLP_H + t] = tiles_done ? r[i] : 0.f;
        }
    }
    __syncthreads();
    if (t < MLP_H) {
        gp[OFF_B1 + t] = gb1[t];
        gp[OFF_B2 + t] = gb2[t];
        gp[OFF_W3 + t] = gw3[t];
    }
    if (t == 0) {
        gp[OFF_B3] = gsc[1];
        gp[MLP_NPARAM] = gsc[0];
        if (!ok) atomicExch(err, 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    tmem_free(tmem_holder, 512);
}

// grad[i] = sum over blocks of part[b][i] in block order (and the loss in grad's tail slot)
__global__ void k_sum_partials(const float* part, int blocks, float* grad, float* loss) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > MLP_NPARAM) return;
    float s = 0.f;
    for (int b = 0; b < blocks; ++b) s += part[(size_t)b * (MLP_NPARAM + 1) + i];
    if (i < MLP_NPARAM) grad[i] = s;
    else loss[0] = s;
}

// ------------------------------------------------------------------ AdamW
__global__ void k_adamw(float* p, const float* g, float* m, float* v, int np, float lr, float b1, float b2, float eps,
                        float wd, float c1, float c2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.f - b1) * gi;
    float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * p[i]);
}

int mlp_grid(int n) {
    int tiles = (n + 127) / 128;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return tiles < sms ? (tiles < 1 ? 1 : tiles) : sms;
}

}  // namespace

extern "C" int vrc_coarse_features(vrc_scene* s, const float* d_pos, int32_t n, const vrc_record_params* p,
                                   float* d_feat, void* stream) {
    if (!s || !p || n < 0) return VRC_ERR_INVALID;
    if (n == 0) return VRC_OK;
    if (!d_pos || !d_feat || p->n_bands < 1 || p->n_bins < 1) return VRC_ERR_INVALID;
    long long items = (long long)n * p->n_bands * p->n_bins;
    int blocks = (int)std::min<long long>((items + 255) / 256, (long long)s->sm_count * 16);
    k_coarse_features<float><<<blocks, 256, 0, (cudaStream_t)stream>>>(s->dev, d_pos, n, p->n_bands, p->n_bins, p->seed,
                                                               p->rec_base, d_feat);
    return cudaGetLastError() == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}

extern "C" int vrc_coarse_features_bf16(vrc_scene* s, const float* d_pos, int32_t n, const vrc_record_params* p,
                                        void* d_feat, void* stream) {
    if (!s || !p || n < 0) return VRC_ERR_INVALID;
    if (n == 0) return VRC_OK;
    if (!d_pos || !d_feat || p->n_bands < 1 || p->n_bins < 1) return VRC_ERR_INVALID;
    long long items = (long long)n * p->n_bands * p->n_bins;
    int blocks = (int)std::min<long long>((items + 255) / 256, (long long)s->sm_count * 16);
    k_coarse_features<__nv_bfloat16><<<blocks, 256, 0, (cudaStream_t)stream>>>(
        s->dev, d_pos, n, p->n_bands, p->n_bins, p->seed, p->rec_base, static_cast<__nv_bfloat16*>(d_feat));
    return cudaGetLastError() == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}

extern "C" int vrc_mlp_create(const float* h_params, vrc_mlp** out) {
    if (!out || !h_params) return VRC_ERR_INVALID;
    *out = nullptr;
    vrc_mlp* m = new vrc_mlp();
    size_t bytes = sizeof(float) * MLP_NPARAM;
    if (cudaMalloc((void**)&m->params, bytes) != cudaSuccess || cudaMalloc((void**)&m->grad, bytes) != cudaSuccess ||
        cudaMalloc((void**)&m->m, bytes) != cudaSuccess || cudaMalloc((void**)&m->v, bytes) != cudaSuccess ||
        cudaMalloc((void**)&m->loss, sizeof(float)) != cudaSuccess ||
        cudaMalloc((void**)&m->err, sizeof(int)) != cudaSuccess) {
        vrc_mlp_destroy(m);
        return VRC_ERR_OOM;
    }
    if (cudaMemcpy(m->params, h_params, bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->m, 0, bytes) != cudaSuccess || cudaMemset(m->v, 0, bytes) != cudaSuccess ||
        cudaMemset(m->err, 0, sizeof(int)) != cudaSuccess) {
        vrc_mlp_destroy(m);
        return VRC_ERR_CUDA;
    }
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, MlpSmem::FWD_END + 1024);
        cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, MlpSmem::END + 1024);
        cudaFuncSetAttribute(k_mlp_forward_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, MlpSmem::FWD_END + 1024);
        attr_set = true;
    }
    *out = m;
    return VRC_OK;
}

extern "C" void vrc_mlp_destroy(vrc_mlp* m) {
    if (!m) return;
    cudaFree(m->params);
    cudaFree(m->grad);
    cudaFree(m->m);
    cudaFree(m->v);
    cudaFree(m->loss);
    cudaFree(m->partial);
    cudaFree(m->err);
    delete m;
}

extern "C" int32_t vrc_mlp_num_params(void) { return MLP_NPARAM; }

extern "C" int vrc_mlp_get_params(const vrc_mlp* m, float* h_params, float* h_adam_m, float* h_adam_v,
                                  int64_t* h_step) {
    if (!m || !h_params) return VRC_ERR_INVALID;
    size_t bytes = sizeof(float) * MLP_NPARAM;
    VRC_CUDA_CHECK(cudaMemcpy(h_params, m->params, bytes, cudaMemcpyDeviceToHost));
    if (h_adam_m) VRC_CUDA_CHECK(cudaMemcpy(h_adam_m, m->m, bytes, cudaMemcpyDeviceToHost));
    if (h_adam_v) VRC_CUDA_CHECK(cudaMemcpy(h_adam_v, m->v, bytes, cudaMemcpyDeviceToHost));
    if (h_step) *h_step = m->step;
    return VRC_OK;
}

extern "C" int vrc_mlp_set_params(vrc_mlp* m, const float* h_params, const float* h_adam_m, const float* h_adam_v,
                                  int64_t step) {
    if (!m || !h_params || step < 0) return VRC_ERR_INVALID;
    size_t bytes = sizeof(float) * MLP_NPARAM;
    VRC_CUDA_CHECK(cudaMemcpy(m->params, h_params, bytes, cudaMemcpyHostToDevice));
    if (h_adam_m) VRC_CUDA_CHECK(cudaMemcpy(m->m, h_adam_m, bytes, cudaMemcpyHostToDevice));
    if (h_adam_v) VRC_CUDA_CHECK(cudaMemcpy(m->v, h_adam_v, bytes, cudaMemcpyHostToDevice));
    m->step = step;
    return VRC_OK;
}

extern "C" int vrc_mlp_predict(const vrc_mlp* m, const float* d_feat, int32_t n, float* d_logr, void* stream) {
    if (!m || n < 0) return VRC_ERR_INVALID;
    if (n == 0) return VRC_OK;
    if (!d_feat || !d_logr) return VRC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(d_feat) & 15) != 0) return VRC_ERR_INVALID;
    int fwd_blocks = mlp_grid(n);
    {
        // two forward blocks fit an SM (106 KB of shared memory, 128 TMEM columns each)
        int tiles = (n + 127) / 128, per2 = 2 * fwd_blocks;
        fwd_blocks = tiles < per2 ? (tiles < 1 ? 1 : tiles) : per2;
    }
    k_mlp_forward<<<fwd_blocks, 128, MlpSmem::FWD_END + 1024, (cudaStream_t)stream>>>(m->params, d_feat, n, d_logr,
                                                                                      m->err);
    return cudaGetLastError() == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to the driver library)
typedef CUresult (*encode_tiled_fn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static encode_tiled_fn encode_tiled() {
    static encode_tiled_fn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<encode_tiled_fn>(p);
    }
    return fn;
}

extern "C" int vrc_mlp_predict_bf16(const vrc_mlp* m, const void* d_feat, int32_t n, float* d_logr, void* stream) {
    if (!m || n < 0) return VRC_ERR_INVALID;
    if (n == 0) return VRC_OK;
    if (!d_feat || !d_logr) return VRC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(d_feat) & 15) != 0) return VRC_ERR_INVALID;   // a TMA source rule
    encode_tiled_fn enc = encode_tiled();
    if (!enc) return VRC_ERR_UNSUPPORTED;
    // [n rows x 256 BF16] row-major; box 64 x 128 with the 128-byte swizzle of the operand layout
    CUtensorMap map;
    cuuint64_t dims[2] = {(cuuint64_t)MLP_IN, (cuuint64_t)n};
    cuuint64_t strides[1] = {(cuuint64_t)MLP_IN * 2};
    cuuint32_t box[2] = {64, 128};
    cuuint32_t estr[2] = {1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(d_feat), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return VRC_ERR_INVALID;
    // two blocks per SM, at most one per tile
    int blocks = mlp_grid(n);
    {
        int tiles = (n + 127) / 128, per2 = 2 * blocks;
        blocks = tiles < per2 ? (tiles < 1 ? 1 : tiles) : per2;
    }
    k_mlp_forward_tma<<<blocks, 128, MlpSmem::FWD_END + 1024, (cudaStream_t)stream>>>(map, m->params, n, d_logr,
                                                                                      m->err);
    return cudaGetLastError() == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}

extern "C" int vrc_mlp_gradient(vrc_mlp* m, const float* d_feat, const float* d_target, int32_t n, float* d_grad,
                                float* d_pred, void* stream) {
    if (!m || n < 1 || !d_feat || !d_target) return VRC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(d_feat) & 15) != 0) return VRC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    float* g = d_grad ? d_grad : m->grad;
    int blocks = mlp_grid(n);
    if (m->partial_blocks < blocks) {
        cudaFree(m->partial);
        m->partial = nullptr;
        m->partial_blocks = 0;
        if (cudaMalloc((void**)&m->partial, sizeof(float) * (size_t)blocks * (MLP_NPARAM + 1)) != cudaSuccess)
            return VRC_ERR_OOM;
        m->partial_blocks = blocks;
    }
    k_mlp_grad<<<blocks, 128, MlpSmem::END + 1024, st>>>(m->params, d_feat, d_target, n, 1.0f / (float)n, m->partial,
                                                         d_pred, m->err);
    k_sum_partials<<<(MLP_NPARAM + 1 + 255) / 256, 256, 0, st>>>(m->partial, blocks, g, m->loss);
    return cudaGetLastError() == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}

extern "C" int vrc_mlp_train_step(vrc_mlp* m, const float* d_feat, const float* d_target, int32_t n, float lr,
                                  float weight_decay, float* h_loss, void* stream) {
    int rc = vrc_mlp_gradient(m, d_feat, d_target, n, nullptr, nullptr, stream);
    if (rc != VRC_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.0f - powf(b1, (float)m->step), c2 = 1.0f - powf(b2, (float)m->step);
    k_adamw<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(m->params, m->grad, m->m, m->v, MLP_NPARAM, lr, b1, b2, 1e-8f,
                                                      weight_decay, c1, c2);
    if (cudaGetLastError() != cudaSuccess) return VRC_ERR_CUDA;
    if (h_loss) {
        float l = 0.f;
        VRC_CUDA_CHECK(cudaMemcpyAsync(&l, m->loss, sizeof(l), cudaMemcpyDeviceToHost, st));
        VRC_CUDA_CHECK(cudaStreamSynchronize(st));
        *h_loss = l / (float)n;
    }
    return VRC_OK;
}

extern "C" int vrc_mlp_status(const vrc_mlp* m) {
    if (!m) return VRC_ERR_INVALID;
    int e = 0;
    VRC_CUDA_CHECK(cudaMemcpy(&e, m->err, sizeof(int), cudaMemcpyDeviceToHost));
    return e ? VRC_ERR_TIMEOUT : VRC_OK;
}
