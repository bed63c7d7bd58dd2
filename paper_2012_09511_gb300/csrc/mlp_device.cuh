// mlp_device.cuh -- the ordering network on tensor cores (not in the paper):
// X [rows][D0] -> relu(X W1 + b1) [H] -> relu(. W2 + b2) [H] -> . W3 + b3 [O],
// bf16 operands and fp32 accumulation with 16x16x16 WMMA tiles, one warp per
// 16-row tile.  Output column 0 is the "descend first" logit of a child row;
// columns 1..P are the machine-pair logits of a parent row.
#pragma once

#include <cuda_bf16.h>
#include <mma.h>

namespace pfsp {

constexpr int kMlpHidden = 128;

struct MlpDev {
    int D0, H, O;                          // input width (3m rounded to 16), hidden, outputs (1+P rounded to 16)
    const __nv_bfloat16 *W1, *W2, *W3;     // [D0][H], [H][H], [H][O] row-major
    const float *b1, *b2, *b3;
};

// One dense layer on a 16-row tile: out = act(A [16][K] x W [K][N] + b).
// A, W bf16 row-major; the result goes to outb (bf16, with ReLU) or outf
// (fp32, no activation); st is a 16x16 fp32 staging tile.
template <bool RELU>
__device__ inline void mlp_dense_tile(const __nv_bfloat16 *A, int K, const __nv_bfloat16 *W, const float *b, int N,
                                      __nv_bfloat16 *outb, float *outf, int ldo, float *st) {
    using namespace nvcuda;
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < N; j += 16) {
        wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc;
        wmma::fill_fragment(acc, 0.0f);
        for (int k = 0; k < K; k += 16) {
            wmma::fragment<wmma::matrix_a, 16, 16, 16, __nv_bfloat16, wmma::row_major> fa;
            wmma::fragment<wmma::matrix_b, 16, 16, 16, __nv_bfloat16, wmma::row_major> fb;
            wmma::load_matrix_sync(fa, A + k, K);
            wmma::load_matrix_sync(fb, W + (size_t)k * N + j, N);
            wmma::mma_sync(acc, fa, fb, acc);
        }
        wmma::store_matrix_sync(st, acc, 16, wmma::mem_row_major);
        __syncwarp();
        for (int e = lane; e < 256; e += 32) {
            const int r = e >> 4, c = e & 15;
            float v = st[e] + b[j + c];
            if (RELU) {
                v = fmaxf(v, 0.0f);
                outb[r * ldo + j + c] = __float2bfloat16_rn(v);
            } else {
                outf[r * ldo + j + c] = v;
            }
        }
        __syncwarp();
    }
}

// Forward pass of one 16-row tile held in shared memory.
__device__ inline void mlp_tile_forward(const MlpDev &P, const __nv_bfloat16 *Xs, __nv_bfloat16 *H1s,
                                        __nv_bfloat16 *H2s, float *st, float *Y, int ldy) {
    mlp_dense_tile<true>(Xs, P.D0, P.W1, P.b1, P.H, H1s, nullptr, P.H, st);
    mlp_dense_tile<true>(H1s, P.H, P.W2, P.b2, P.H, H2s, nullptr, P.H, st);
    mlp_dense_tile<false>(H2s, P.H, P.W3, P.b3, P.O, nullptr, Y, ldy, st);
}

// ---- fused inference: the three layers of a 16-row tile in registers --------
// mma.sync m16n8k16 (bf16 in, fp32 accumulate): the accumulator fragment of
// output columns 16p..16p+15 (n-tiles 2p and 2p+1) holds, per thread, exactly
// the elements of the next layer's A fragment for k-tile p (rows g and g + 8,
// columns 2t, 2t + 1 and 8 + 2t, 9 + 2t, g = lane / 4, t = lane % 4), so bias,
// ReLU and the bf16 rounding are applied in registers and no activation goes
// through memory.  B fragments are read by each thread straight from the
// image in global memory through the read-only path (the image, about 50 KB,
// stays in L1/L2; staging it in shared memory would cost explorer warps).
//
// The image (in global memory, built by mlp_build_image):
// W1t [H][D0 + 8], W2t [H][H + 8], W3t [O3][H + 8] bf16, transposed ([out][in])
// with rows padded by 8 elements; then b1 [H], b2 [H], b3 [O3] fp32.  Every
// row and every bias array starts on an 8-byte boundary.
// O3 (a multiple of 16) output columns are staged: 16 when only the
// descend-first logit (column 0) is needed, O for the pair head too.
struct MlpImage {
    const __nv_bfloat16 *W1t, *W2t, *W3t;
    const float *b1, *b2, *b3;
    int D0, O3;
};

__host__ __device__ inline int mlp_image_bytes(int D0, int O3) {
    const int H = kMlpHidden;
    return 2 * (H * (D0 + 8) + H * (H + 8) + O3 * (H + 8)) + 4 * (2 * H + O3);
}

__host__ __device__ inline MlpImage mlp_image_view(const void *base, int D0, int O3) {
    const int H = kMlpHidden;
    MlpImage P;
    P.D0 = D0;
    P.O3 = O3;
    P.W1t = reinterpret_cast<const __nv_bfloat16 *>(base);
    P.W2t = P.W1t + H * (D0 + 8);
    P.W3t = P.W2t + H * (H + 8);
    P.b1 = reinterpret_cast<const float *>(P.W3t + O3 * (H + 8));
    P.b2 = P.b1 + H;
    P.b3 = P.b2 + H;
    return P;
}

// Per-warp scratch of fused inference, bf16 tiles of 16 rows: the input Xs
// [16][D0 + 8], layer 1's activations H1 [16][H + 8] and layer 2's H2
// [16][H + 8] (kept only for the pair head).
__host__ __device__ inline int mlp_scratch_bytes(int D0) { return 32 * (D0 + 8) + 64 * (kMlpHidden + 8); }

__device__ __forceinline__ unsigned mlp_pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<unsigned *>(&v);
}

__device__ __forceinline__ void mlp_mma(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mlp_ldsm4(unsigned (&r)[4], const __nv_bfloat16 *row) {
    const unsigned addr = (unsigned)__cvta_generic_to_shared(row);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

// B fragments of k-tile kk for the n-tiles 16p..16p+7 (b[0], b[1]) and
// 16p+8..16p+15 (b[2], b[3]) of transposed weights Wt [N][ldw] in global
// memory: thread (g, t) takes the bf16 pairs at columns 16kk + 2t and
// 16kk + 8 + 2t of rows 16p + g and 16p + 8 + g.
__device__ __forceinline__ void mlp_ldg_b4(unsigned (&b)[4], const __nv_bfloat16 *Wt, int ldw, int p, int kk) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const unsigned *r0 = reinterpret_cast<const unsigned *>(Wt + (size_t)(16 * p + g) * ldw + 16 * kk + 2 * t);
    const unsigned *r1 = r0 + 4 * ldw;  // 8 rows further (ldw bf16 = ldw / 2 words per row)
    b[0] = __ldg(r0);
    b[1] = __ldg(r0 + 4);
    b[2] = __ldg(r1);
    b[3] = __ldg(r1 + 4);
}

// Raw products (no bias) for output columns 16p..16p+15 of a 16-row tile
// whose KT k-tiles of input come from the shared tile As ([16][lda] bf16,
// one ldmatrix per k-tile): c0 holds columns 16p + 2t, +1 and c1 columns
// 16p + 8 + 2t, +1, of rows g ([0], [1]) and g + 8 ([2], [3]).
// Wt: [N][ldw] transposed weights in global memory.
template <int KT>
__device__ __forceinline__ void mlp_tile_cols(const __nv_bfloat16 *As, int lda, const __nv_bfloat16 *Wt, int ldw,
                                              int p, float (&c0)[4], float (&c1)[4]) {
    const int lane = threadIdx.x & 31, q = lane >> 3, r = lane & 7;
    const __nv_bfloat16 *x = As + (r + 8 * (q & 1)) * lda + 8 * (q >> 1);
#pragma unroll
    for (int i = 0; i < 4; ++i) c0[i] = c1[i] = 0.0f;
#pragma unroll
    for (int kk = 0; kk < KT; ++kk) {
        unsigned av[4], b[4];
        mlp_ldsm4(av, x + 16 * kk);
        mlp_ldg_b4(b, Wt, ldw, p, kk);
        mlp_mma(c0, av, b[0], b[1]);
        mlp_mma(c1, av, b[2], b[3]);
    }
}

// One hidden layer on a shared input tile: relu(A W + b) rounded to bf16.
// Output k-tile p (the next layer's A fragment for columns 16p..16p+15) goes
// to sink(p, frag) as soon as it is computed; the loop over p stays rolled,
// so only a few fragments are live at a time.
template <int KT, class Sink>
__device__ __forceinline__ void mlp_layer_relu(const __nv_bfloat16 *As, int lda, const __nv_bfloat16 *Wt, int ldw,
                                               const float *b, Sink &&sink) {
    const int t = threadIdx.x & 3;
#pragma unroll 1
    for (int p = 0; p < kMlpHidden / 16; ++p) {
        float c0[4], c1[4];
        mlp_tile_cols<KT>(As, lda, Wt, ldw, p, c0, c1);
        const float2 e0 = __ldg(reinterpret_cast<const float2 *>(b + 16 * p + 2 * t));
        const float2 e1 = __ldg(reinterpret_cast<const float2 *>(b + 16 * p + 8 + 2 * t));
        unsigned o[4];
        o[0] = mlp_pack_bf16(fmaxf(c0[0] + e0.x, 0.0f), fmaxf(c0[1] + e0.y, 0.0f));
        o[1] = mlp_pack_bf16(fmaxf(c0[2] + e0.x, 0.0f), fmaxf(c0[3] + e0.y, 0.0f));
        o[2] = mlp_pack_bf16(fmaxf(c1[0] + e1.x, 0.0f), fmaxf(c1[1] + e1.y, 0.0f));
        o[3] = mlp_pack_bf16(fmaxf(c1[2] + e1.x, 0.0f), fmaxf(c1[3] + e1.y, 0.0f));
        sink(p, o);
    }
}

// A sink that parks a layer's activations in a shared tile [16][H + 8] bf16
// (row-major, the layout ldmatrix reads back as A fragments).
struct MlpPark {
    __nv_bfloat16 *Hs;
    __device__ __forceinline__ void operator()(int p, const unsigned (&o)[4]) const {
        const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
        const int ld = kMlpHidden + 8;
        unsigned *r0 = reinterpret_cast<unsigned *>(Hs + g * ld + 16 * p + 2 * t);
        unsigned *r1 = reinterpret_cast<unsigned *>(Hs + (g + 8) * ld + 16 * p + 2 * t);
        r0[0] = o[0];
        r1[0] = o[1];
        r0[4] = o[2];  // columns + 8
        r1[4] = o[3];
    }
};

// A sink that runs layer 3 for output columns 0..7 on the fly: acc holds the
// raw logits of columns 2t, 2t + 1 of rows g ([0], [1]) and g + 8 ([2], [3]).
struct MlpFirstCols {
    const __nv_bfloat16 *W3t;
    float (&acc)[4];
    __device__ __forceinline__ void operator()(int p, const unsigned (&o)[4]) const {
        const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
        const unsigned *r = reinterpret_cast<const unsigned *>(W3t + g * (kMlpHidden + 8) + 16 * p + 2 * t);
        mlp_mma(acc, o, __ldg(r), __ldg(r + 4));
    }
};

// Layers 1 and 2 of the tile Xs ([16][D0 + 8], KT1 = D0 / 16): layer 1's
// activations are parked in H1, layer 2's handed to sink(p, frag).
template <int KT1, class Sink>
__device__ __forceinline__ void mlp_fused_hidden(const MlpImage &P, const __nv_bfloat16 *Xs, __nv_bfloat16 *H1,
                                                 Sink &&sink) {
    mlp_layer_relu<KT1>(Xs, 16 * KT1 + 8, P.W1t, 16 * KT1 + 8, P.b1, MlpPark{H1});
    __syncwarp();
    mlp_layer_relu<kMlpHidden / 16>(H1, kMlpHidden + 8, P.W2t, kMlpHidden + 8, P.b2, sink);
    __syncwarp();
}

}  // namespace pfsp
