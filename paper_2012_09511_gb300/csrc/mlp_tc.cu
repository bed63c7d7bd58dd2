// mlp_tc.cu -- batched forward pass of the ordering network (not in the
// paper) on the fifth-generation tensor cores: tcgen05.mma with operands in
// shared memory and fp32 accumulators in tensor memory (TMEM).
//
// One CTA of 128 threads runs 128-row tiles (the MMA's M): the tile of
// inputs X [128][D0] and the transposed weights W1^T [128][D0], W2^T
// [128][128], W3^T [O][128] sit in shared memory as bf16 in the K-major
// layout without swizzle (8 x 8 core matrices of 128 contiguous bytes, the
// cores adjacent in K 128 bytes apart, the 8-row groups K/8 x 128 bytes
// apart).  One elected thread issues each layer's MMAs (K/16 instructions of
// 128 x N x 16) into TMEM columns 0..N-1 and commits them to an mbarrier;
// after the bounded wait every thread reads its own row (TMEM lane = row)
// with tcgen05.ld, adds the bias, applies ReLU, rounds to bf16 and writes the
// row into the next layer's operand tile.  The last layer's row goes to Y
// with its bias, in fp32.  This is the network of mlp_device.cuh (bf16
// operands, fp32 accumulation), so results agree with it up to the order of
// the fp32 sums.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mlp_device.cuh"
#include "pfsp_internal.h"

namespace pfsp {

constexpr int kTcRows = 128;                // rows per tile: the MMA's M, one TMEM lane per row
constexpr int kTcThreads = 128;             // one thread per row
constexpr int kTcTmemCols = 256;            // accumulator columns allocated (a power of two >= H, O)
constexpr long long kTcWaitLimit = 1 << 24;  // polls of an mbarrier before the kernel gives up

static __device__ int g_mlp_tc_err;  // nonzero: a bounded wait expired (host reads and clears it)

// Byte offset of element (r, k) of a K-major operand tile with K columns.
__device__ __forceinline__ uint32_t tc_off(int r, int k, int K) {
    return (uint32_t)((r >> 3) * (K >> 3) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor: start address, leading byte offset (the
// next core matrix along K: 128 bytes), stride byte offset (the next 8-row
// group: K/8 x 128 bytes), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, int K) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)(128u >> 4) << 16;
    d |= (uint64_t)((((uint32_t)K >> 3) * 128u >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: D fp32, A and B bf16, both K-major,
// N columns, M = 128 rows.
__host__ __device__ constexpr uint32_t tc_idesc(int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// D[128][N] (TMEM columns 0..N-1) = A[128][K] x B[N][K]^T, issued by one thread
// and committed to the mbarrier.
__device__ __forceinline__ void tc_layer(uint32_t tmem, uint32_t sa, uint32_t sb, int K, int N, uint32_t bar) {
    const uint32_t idesc = tc_idesc(N);
    for (int kk = 0; kk < K / 16; ++kk) {
        const uint64_t da = tc_desc(sa + kk * 256u, K), db = tc_desc(sb + kk * 256u, K);
        const uint32_t acc = kk > 0 ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc)
            : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// Bounded wait for the mbarrier phase `parity`; false when the limit ran out.
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) {
    for (long long it = 0; it < kTcWaitLimit; ++it) {
        uint32_t ready = 0;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ready)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ready) return true;
    }
    return false;
}

// 16 consecutive fp32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Hidden-layer epilogue: row `row` of the accumulators (128 columns) plus
// bias, ReLU, bf16, into the next operand tile (K = 128).
__device__ __forceinline__ void tc_hidden_epilogue(uint32_t tlane, const float *bias, unsigned char *next, int row) {
#pragma unroll 1
    for (int c0 = 0; c0 < kMlpHidden; c0 += 16) {
        float v[16];
        tc_ld16(tlane + (uint32_t)c0, v);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            __align__(16) __nv_bfloat16 b[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) b[i] = __float2bfloat16_rn(fmaxf(v[8 * h + i] + bias[c0 + 8 * h + i], 0.0f));
            *reinterpret_cast<uint4 *>(next + tc_off(row, c0 + 8 * h, kMlpHidden)) = *reinterpret_cast<uint4 *>(b);
        }
    }
}

// Shared-memory layout of the kernel (bytes; every region 1024-aligned).
struct TcSmem {
    uint32_t a1, a2, b1, b2, b3, bias, bar, total;
};

__host__ __device__ inline TcSmem tc_smem(int D0, int O) {
    TcSmem s;
    uint32_t o = 0;
    auto take = [&](uint32_t bytes) {
        uint32_t r = o;
        o = (o + bytes + 1023u) & ~1023u;
        return r;
    };
    s.a1 = take(kTcRows * D0 * 2);
    s.a2 = take(kTcRows * kMlpHidden * 2);
    s.b1 = take(kMlpHidden * D0 * 2);
    s.b2 = take(kMlpHidden * kMlpHidden * 2);
    s.b3 = take(O * kMlpHidden * 2);
    s.bias = take((2 * kMlpHidden + O) * 4);
    s.bar = take(16);
    s.total = o;
    return s;
}

__global__ void __launch_bounds__(kTcThreads, 1) mlp_forward_tc_kernel(MlpDev P, const float *X, long long rows,
                                                                       float *Y) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int D0 = P.D0, O = P.O, H = kMlpHidden;
    const TcSmem L = tc_smem(D0, O);
    const int tid = threadIdx.x, warp = tid >> 5;
    unsigned char *A1 = sm + L.a1, *A2 = sm + L.a2, *B1 = sm + L.b1, *B2 = sm + L.b2, *B3 = sm + L.b3;
    float *bias = reinterpret_cast<float *>(sm + L.bias);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + L.bar);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(sm + L.bar + 8);
    const uint32_t sbar = smem_u32(bar);

    // transposed bf16 weights and fp32 biases, once per CTA
    for (int e = tid; e < H * D0; e += kTcThreads) {
        const int n = e / D0, k = e % D0;
        *reinterpret_cast<__nv_bfloat16 *>(B1 + tc_off(n, k, D0)) = P.W1[(size_t)k * H + n];
    }
    for (int e = tid; e < H * H; e += kTcThreads) {
        const int n = e / H, k = e % H;
        *reinterpret_cast<__nv_bfloat16 *>(B2 + tc_off(n, k, H)) = P.W2[(size_t)k * H + n];
    }
    for (int e = tid; e < O * H; e += kTcThreads) {
        const int n = e / H, k = e % H;
        *reinterpret_cast<__nv_bfloat16 *>(B3 + tc_off(n, k, H)) = P.W3[(size_t)k * O + n];
    }
    for (int e = tid; e < 2 * H + O; e += kTcThreads)
        bias[e] = e < H ? P.b1[e] : (e < 2 * H ? P.b2[e - H] : P.b3[e - 2 * H]);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sbar));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(kTcTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_holder;
    // this thread's TMEM lane (its row of the tile), column 0
    const uint32_t tlane = tmem + ((uint32_t)(warp * 32) << 16);
    const uint32_t sa1 = smem_u32(A1), sa2 = smem_u32(A2), sb1 = smem_u32(B1), sb2 = smem_u32(B2),
                   sb3 = smem_u32(B3);

    uint32_t phase = 0;
    bool ok = true;
    const long long tiles = (rows + kTcRows - 1) / kTcRows;
    for (long long tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const long long r = tile * kTcRows + tid;
        // this thread's input row, bf16, into the first operand tile
        for (int k0 = 0; k0 < D0; k0 += 8) {
            __align__(16) __nv_bfloat16 b[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) b[i] = __float2bfloat16_rn(r < rows ? X[r * D0 + k0 + i] : 0.0f);
            *reinterpret_cast<uint4 *>(A1 + tc_off(tid, k0, D0)) = *reinterpret_cast<uint4 *>(b);
        }
        // three layers: operands written by the threads are made visible to
        // the tensor cores (async proxy) before the elected thread issues
#pragma unroll 1
        for (int layer = 0; layer < 3 && ok; ++layer) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (layer == 0) tc_layer(tmem, sa1, sb1, D0, H, sbar);
                else if (layer == 1) tc_layer(tmem, sa2, sb2, H, H, sbar);
                else tc_layer(tmem, sa2, sb3, H, O, sbar);
            }
            ok = tc_wait(sbar, phase);
            phase ^= 1u;
            if (!__syncthreads_and(ok)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (layer < 2) {
                // the next operand reuses A2: layer 2's MMAs (which read it)
                // have completed
                tc_hidden_epilogue(tlane, bias + layer * H, A2, tid);
            } else {
                // every thread of the warp runs the same loads (they are
                // warp-collective); only rows of the input are stored
#pragma unroll 1
                for (int c0 = 0; c0 < O; c0 += 16) {
                    float v[16];
                    tc_ld16(tlane + (uint32_t)c0, v);
                    if (r < rows) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) Y[r * O + c0 + i] = v[i] + bias[2 * H + c0 + i];
                    }
                }
            }
        }
    }
    if (!ok && tid == 0) atomicExch(&g_mlp_tc_err, 1);
    // a wait that gave up: give the MMAs in flight one more bounded wait
    // before the accumulators are released
    if (!ok && tid == 0) tc_wait(sbar, phase);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols));
    }
    if (tid == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(sbar) : "memory");
}

// Logits Y [rows][O] of device inputs X [rows][D0] (asynchronous on st);
// *timed_out (host) is set after the stream completes when a bounded wait
// of the kernel expired.
cudaError_t mlp_forward_tc(const MlpDev &P, const float *dX, long long rows, float *dY, cudaStream_t st,
                           bool *timed_out) {
    *timed_out = false;
    if (rows <= 0) return cudaSuccess;
    if (P.H != kMlpHidden || P.D0 % 16 || P.O % 16 || P.O < 16 || P.O > kTcTmemCols || P.D0 > 256)
        return cudaErrorInvalidValue;
    const TcSmem L = tc_smem(P.D0, P.O);
    cudaError_t e = cudaFuncSetAttribute(mlp_forward_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L.total);
    if (e != cudaSuccess) return e;
    int zero = 0, dev = 0, nsm = 1;
    e = cudaMemcpyToSymbolAsync(g_mlp_tc_err, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long tiles = (rows + kTcRows - 1) / kTcRows;
    const int grid = (int)(tiles < nsm ? tiles : nsm);
    mlp_forward_tc_kernel<<<grid, kTcThreads, L.total, st>>>(P, dX, rows, dY);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int err = 0;
    e = cudaMemcpyFromSymbolAsync(&err, g_mlp_tc_err, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    *timed_out = err != 0;
    return e;
}

}  // namespace pfsp
