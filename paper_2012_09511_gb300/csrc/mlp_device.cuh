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

// Per-warp scratch of in-solver inference: Xs [16][D0] bf16, H1s and H2s
// [16][H] bf16, a 16x16 fp32 staging tile (byte offsets, 32-byte aligned).
__host__ __device__ inline int mlp_scratch_bytes(int D0) { return 32 * D0 + 4 * 16 * kMlpHidden + 1024; }

// Layers 1 and 2 of the 16-row tile in Xs; leaves H2s.
__device__ inline void mlp_tile_hidden(const MlpDev &P, unsigned char *ms) {
    __nv_bfloat16 *Xs = (__nv_bfloat16 *)ms;
    __nv_bfloat16 *H1s = (__nv_bfloat16 *)(ms + 32 * P.D0);
    __nv_bfloat16 *H2s = H1s + 16 * P.H;
    float *st = (float *)(H2s + 16 * P.H);
    mlp_dense_tile<true>(Xs, P.D0, P.W1, P.b1, P.H, H1s, nullptr, P.H, st);
    mlp_dense_tile<true>(H1s, P.H, P.W2, P.b2, P.H, H2s, nullptr, P.H, st);
}

// Logits of output columns j..j+15 (without bias) for the 16 rows, left in
// the staging tile (row-major 16 x 16); returns the staging tile.
__device__ inline float *mlp_tile_logits(const MlpDev &P, unsigned char *ms, int j) {
    using namespace nvcuda;
    __nv_bfloat16 *H2s = (__nv_bfloat16 *)(ms + 32 * P.D0) + 16 * P.H;
    float *st = (float *)(H2s + 16 * P.H);
    wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc;
    wmma::fill_fragment(acc, 0.0f);
    for (int k = 0; k < P.H; k += 16) {
        wmma::fragment<wmma::matrix_a, 16, 16, 16, __nv_bfloat16, wmma::row_major> fa;
        wmma::fragment<wmma::matrix_b, 16, 16, 16, __nv_bfloat16, wmma::row_major> fb;
        wmma::load_matrix_sync(fa, H2s + k, P.H);
        wmma::load_matrix_sync(fb, P.W3 + (size_t)k * P.O + j, P.O);
        wmma::mma_sync(acc, fa, fb, acc);
    }
    wmma::store_matrix_sync(st, acc, 16, wmma::mem_row_major);
    __syncwarp();
    return st;
}

}  // namespace pfsp
