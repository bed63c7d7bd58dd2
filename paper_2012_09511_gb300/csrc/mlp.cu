// mlp.cu -- the ordering network (not in the paper): parameters, forward,
// masked binary cross-entropy gradients and Adam training, all on the GPU
// with hand-written kernels (bf16 WMMA tensor-core tiles, fp32 accumulation).
//
// Rows are independent: a parent row carries pair targets (does machine pair
// k,l attain the LB2 maximum of some child?), a child row carries the
// "descend first" target; the mask selects which outputs of a row are
// trained.  Loss = sum_r,o M[r,o] bce(Y[r,o], T[r,o]) / rows.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <mma.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "mlp_device.cuh"
#include "pfsp_internal.h"

struct pfsp_mlp {
    int m, P, D0, H, O;
    int device;
    size_t n_params;
    size_t oW1, ob1, oW2, ob2, oW3, ob3;  // offsets in the fp32 parameter vector
    float *params, *grads, *adam_m, *adam_v;
    __nv_bfloat16 *wb;                    // bf16 copies: W1 | W2 | W3
    long long step;
};

namespace pfsp {

cudaError_t mlp_forward_tc(const MlpDev &P, const float *dX, long long rows, float *dY, cudaStream_t st,
                           bool *timed_out);

static inline int round16(int x) { return (x + 15) & ~15; }

MlpDev mlp_view(const pfsp_mlp *M) {
    MlpDev P;
    P.D0 = M->D0;
    P.H = M->H;
    P.O = M->O;
    P.W1 = M->wb;
    P.W2 = M->wb + (size_t)M->D0 * M->H;
    P.W3 = M->wb + (size_t)M->D0 * M->H + (size_t)M->H * M->H;
    P.b1 = M->params + M->ob1;
    P.b2 = M->params + M->ob2;
    P.b3 = M->params + M->ob3;
    return P;
}

int mlp_dims(const pfsp_mlp *M, int *m, int *D0, int *O) {
    *m = M->m;
    *D0 = M->D0;
    *O = M->O;
    return PFSP_OK;
}

__global__ void mlp_refresh_bf16(const float *params, size_t oW1, size_t nW1, size_t oW2, size_t nW2, size_t oW3,
                                 size_t nW3, __nv_bfloat16 *wb) {
    size_t tot = nW1 + nW2 + nW3;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x) {
        float v = i < nW1 ? params[oW1 + i] : (i < nW1 + nW2 ? params[oW2 + i - nW1] : params[oW3 + i - nW1 - nW2]);
        wb[i] = __float2bfloat16_rn(v);
    }
}

// Per-warp shared-memory layout of the training kernel (bytes, 32-aligned).
struct GradSmem {
    int xs, h1, h2, dy, yf, dh2, dh1, st, total;
};

__host__ __device__ inline GradSmem grad_smem(int D0, int H, int O) {
    GradSmem g;
    int o = 0;
    auto take = [&](int bytes) {
        int r = o;
        o += (bytes + 127) & ~127;
        return r;
    };
    g.xs = take(16 * D0 * 2);
    g.h1 = take(16 * H * 2);
    g.h2 = take(16 * H * 2);
    g.dy = take(16 * O * 2);
    g.yf = take(16 * O * 4);
    g.dh2 = take(16 * H * 2);
    g.dh1 = take(16 * H * 2);
    g.st = take(256 * 4);
    g.total = o;
    return g;
}

// The inference image (layout in mlp_device.cuh) of O3 output columns:
// transposed, row-padded bf16 weights from the bf16 copies, fp32 biases.
__global__ void mlp_image_kernel(MlpDev P, int O3, unsigned char *img) {
    const int H = P.H, D0 = P.D0, O = P.O;
    MlpImage I = mlp_image_view(img, D0, O3);
    __nv_bfloat16 *W1t = const_cast<__nv_bfloat16 *>(I.W1t), *W2t = const_cast<__nv_bfloat16 *>(I.W2t),
                  *W3t = const_cast<__nv_bfloat16 *>(I.W3t);
    float *b1 = const_cast<float *>(I.b1), *b2 = const_cast<float *>(I.b2), *b3 = const_cast<float *>(I.b3);
    const int n1 = H * (D0 + 8), n2 = H * (H + 8), n3 = O3 * (H + 8);
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n1 + n2 + n3 + 2 * H + O3; i += gridDim.x * blockDim.x) {
        if (i < n1) {
            const int o = i / (D0 + 8), k = i % (D0 + 8);
            W1t[i] = k < D0 ? P.W1[k * H + o] : zero;
        } else if (i < n1 + n2) {
            const int o = (i - n1) / (H + 8), k = (i - n1) % (H + 8);
            W2t[i - n1] = k < H ? P.W2[k * H + o] : zero;
        } else if (i < n1 + n2 + n3) {
            const int o = (i - n1 - n2) / (H + 8), k = (i - n1 - n2) % (H + 8);
            W3t[i - n1 - n2] = (k < H && o < O) ? P.W3[k * O + o] : zero;
        } else {
            const int j = i - n1 - n2 - n3;
            if (j < H) b1[j] = P.b1[j];
            else if (j < 2 * H) b2[j - H] = P.b2[j - H];
            else b3[j - 2 * H] = (j - 2 * H) < O ? P.b3[j - 2 * H] : 0.0f;
        }
    }
}

cudaError_t mlp_build_image(const pfsp_mlp *M, int O3, void *dst, cudaStream_t st) {
    const int total = mlp_image_bytes(M->D0, O3) / 2;
    mlp_image_kernel<<<(total + 255) / 256, 256, 0, st>>>(mlp_view(M), O3, (unsigned char *)dst);
    return cudaGetLastError();
}

// Gradients of the masked mean BCE over the batch rows idx[row0 .. row0+n)
// (or rows row0.. when idx is NULL), accumulated into g (same layout as the
// parameters) with atomics; the batch loss is added to *loss.
__global__ void mlp_grad_kernel(MlpDev P, const float *X, const float *T, const float *Mk, const int *idx,
                                long long row0, int n, float inv_rows, float *g, size_t oW1, size_t ob1, size_t oW2,
                                size_t ob2, size_t oW3, size_t ob3, float *loss) {
    using namespace nvcuda;
    extern __shared__ __align__(128) unsigned char sm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int D0 = P.D0, H = P.H, O = P.O;
    GradSmem L = grad_smem(D0, H, O);
    unsigned char *w = sm + (size_t)wib * L.total;
    __nv_bfloat16 *Xs = (__nv_bfloat16 *)(w + L.xs), *H1 = (__nv_bfloat16 *)(w + L.h1), *H2 = (__nv_bfloat16 *)(w + L.h2);
    __nv_bfloat16 *dY = (__nv_bfloat16 *)(w + L.dy), *dH2 = (__nv_bfloat16 *)(w + L.dh2), *dH1 = (__nv_bfloat16 *)(w + L.dh1);
    float *Yf = (float *)(w + L.yf), *st = (float *)(w + L.st);
    const int tiles = (n + 15) / 16;
    const int nw = gridDim.x * (blockDim.x >> 5);
    float my_loss = 0.0f;
    for (int t = blockIdx.x * (blockDim.x >> 5) + wib; t < tiles; t += nw) {
        // rows of this tile (16, the tail padded with zero rows and zero mask)
        for (int e = lane; e < 16 * D0; e += 32) {
            int r = t * 16 + e / D0;
            float v = 0.0f;
            if (r < n) {
                long long src = idx ? idx[row0 + r] : row0 + r;
                v = X[src * D0 + e % D0];
            }
            Xs[e] = __float2bfloat16_rn(v);
        }
        __syncwarp();
        mlp_tile_forward(P, Xs, H1, H2, st, Yf, O);
        // dY = mask * (sigmoid(y) - t) / rows; loss; bias gradient of layer 3
        for (int e = lane; e < 16 * O; e += 32) {
            int r = t * 16 + e / O, c = e % O;
            float d = 0.0f;
            if (r < n) {
                long long src = idx ? idx[row0 + r] : row0 + r;
                float tv = T[src * O + c], mk = Mk[src * O + c], y = Yf[e];
                float s = 1.0f / (1.0f + expf(-y));
                d = mk * (s - tv) * inv_rows;
                my_loss += mk * (fmaxf(y, 0.0f) - y * tv + log1pf(expf(-fabsf(y)))) * inv_rows;
            }
            Yf[e] = d;
            dY[e] = __float2bfloat16_rn(d);
        }
        __syncwarp();
        for (int c = lane; c < O; c += 32) {
            float s = 0.0f;
            for (int r = 0; r < 16; ++r) s += Yf[r * O + c];
            if (s != 0.0f) atomicAdd(g + ob3 + c, s);
        }
        __syncwarp();
        // dW3 = H2^T dY
        for (int hu = 0; hu < H; hu += 16)
            for (int o = 0; o < O; o += 16) {
                wmma::fragment<wmma::matrix_a, 16, 16, 16, __nv_bfloat16, wmma::col_major> fa;
                wmma::fragment<wmma::matrix_b, 16, 16, 16, __nv_bfloat16, wmma::row_major> fb;
                wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc;
                wmma::fill_fragment(acc, 0.0f);
                wmma::load_matrix_sync(fa, H2 + hu, H);
                wmma::load_matrix_sync(fb, dY + o, O);
                wmma::mma_sync(acc, fa, fb, acc);
                wmma::store_matrix_sync(st, acc, 16, wmma::mem_row_major);
                __syncwarp();
                for (int e = lane; e < 256; e += 32) atomicAdd(g + oW3 + (size_t)(hu + (e >> 4)) * O + o + (e & 15), st[e]);
                __syncwarp();
            }
        // dH2 = (dY W3^T) * relu'(H2); bias gradient of layer 2
        for (int j = 0; j < H; j += 16) {
            wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc;
            wmma::fill_fragment(acc, 0.0f);
            for (int o = 0; o < O; o += 16) {
                wmma::fragment<wmma::matrix_a, 16, 16, 16, __nv_bfloat16, wmma::row_major> fa;
                wmma::fragment<wmma::matrix_b, 16, 16, 16, __nv_bfloat16, wmma::col_major> fb;
                wmma::load_matrix_sync(fa, dY + o, O);
                wmma::load_matrix_sync(fb, P.W3 + (size_t)j * O + o, O);
                wmma::mma_sync(acc, fa, fb, acc);
            }
            wmma::store_matrix_sync(st, acc, 16, wmma::mem_row_major);
            __syncwarp();
            for (int e = lane; e < 256; e += 32) {
                int r = e >> 4, c = e & 15;
                float v = __bfloat162float(H2[r * H + j + c]) > 0.0f ? st[e] : 0.0f;
                st[e] = v;
                dH2[r * H + j + c] = __float2bfloat16_rn(v);
            }
            __syncwarp();
            if (lane < 16) {
                float s = 0.0f;
                for (int r = 0; r < 16; ++r) s += st[r * 16 + lane];
                if (s != 0.0f) atomicAdd(g + ob2 + j + lane, s);
            }
            __syncwarp();
        }
        // dW2 = H1^T dH2
        for (int hu = 0; hu < H; hu += 16)
            for (int j = 0; j < H; j += 16) {
                wmma::fragment<wmma::matrix_a, 16, 16, 16, __nv_bfloat16, wmma::col_major> fa;
                wmma::fragment<wmma::matrix_b, 16, 16, 16, __nv_bfloat16, wmma::row_major> fb;
                wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc;
                wmma::fill_fragment(acc, 0.0f);
                wmma::load_matrix_sync(fa, H1 + hu, H);
                wmma::load_matrix_sync(fb, dH2 + j, H);
                wmma::mma_sync(acc, fa, fb, acc);
                wmma::store_matrix_sync(st, acc, 16, wmma::mem_row_major);
                __syncwarp();
                for (int e = lane; e < 256; e += 32) atomicAdd(g + oW2 + (size_t)(hu + (e >> 4)) * H + j + (e & 15), st[e]);
                __syncwarp();
            }
        // dH1 = (dH2 W2^T) * relu'(H1); bias gradient of layer 1
        for (int j = 0; j < H; j += 16) {
            wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc;
            wmma::fill_fragment(acc, 0.0f);
            for (int k = 0; k < H; k += 16) {
                wmma::fragment<wmma::matrix_a, 16, 16, 16, __nv_bfloat16, wmma::row_major> fa;
                wmma::fragment<wmma::matrix_b, 16, 16, 16, __nv_bfloat16, wmma::col_major> fb;
                wmma::load_matrix_sync(fa, dH2 + k, H);
                wmma::load_matrix_sync(fb, P.W2 + (size_t)j * H + k, H);
                wmma::mma_sync(acc, fa, fb, acc);
            }
            wmma::store_matrix_sync(st, acc, 16, wmma::mem_row_major);
            __syncwarp();
            for (int e = lane; e < 256; e += 32) {
                int r = e >> 4, c = e & 15;
                float v = __bfloat162float(H1[r * H + j + c]) > 0.0f ? st[e] : 0.0f;
                st[e] = v;
                dH1[r * H + j + c] = __float2bfloat16_rn(v);
            }
            __syncwarp();
            if (lane < 16) {
                float s = 0.0f;
                for (int r = 0; r < 16; ++r) s += st[r * 16 + lane];
                if (s != 0.0f) atomicAdd(g + ob1 + j + lane, s);
            }
            __syncwarp();
        }
        // dW1 = X^T dH1
        for (int d = 0; d < D0; d += 16)
            for (int j = 0; j < H; j += 16) {
                wmma::fragment<wmma::matrix_a, 16, 16, 16, __nv_bfloat16, wmma::col_major> fa;
                wmma::fragment<wmma::matrix_b, 16, 16, 16, __nv_bfloat16, wmma::row_major> fb;
                wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc;
                wmma::fill_fragment(acc, 0.0f);
                wmma::load_matrix_sync(fa, Xs + d, D0);
                wmma::load_matrix_sync(fb, dH1 + j, H);
                wmma::mma_sync(acc, fa, fb, acc);
                wmma::store_matrix_sync(st, acc, 16, wmma::mem_row_major);
                __syncwarp();
                for (int e = lane; e < 256; e += 32) atomicAdd(g + oW1 + (size_t)(d + (e >> 4)) * H + j + (e & 15), st[e]);
                __syncwarp();
            }
    }
    for (int o = 16; o; o >>= 1) my_loss += __shfl_xor_sync(0xffffffffu, my_loss, o);
    if (lane == 0 && my_loss != 0.0f) atomicAdd(loss, my_loss);
}

// Adam (Kingma & Ba) on the fp32 parameters; the gradients are cleared.
__global__ void mlp_adam_kernel(float *p, float *g, float *m1, float *m2, size_t n, float lr, float b1, float b2,
                                float eps, float c1, float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float gi = g[i];
        float a = b1 * m1[i] + (1.0f - b1) * gi;
        float v = b2 * m2[i] + (1.0f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = v;
        p[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
        g[i] = 0.0f;
    }
}

static cudaError_t refresh(pfsp_mlp *M) {
    size_t nW1 = (size_t)M->D0 * M->H, nW2 = (size_t)M->H * M->H, nW3 = (size_t)M->H * M->O;
    mlp_refresh_bf16<<<64, 256>>>(M->params, M->oW1, nW1, M->oW2, nW2, M->oW3, nW3, M->wb);
    return cudaGetLastError();
}

static int grad_blocks_and_smem(const pfsp_mlp *M, int warps, size_t *smem) {
    GradSmem L = grad_smem(M->D0, M->H, M->O);
    *smem = (size_t)L.total * warps;
    cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return nsm;
}

static uint64_t splitmix(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace pfsp

using namespace pfsp;

namespace pfsp {

}  // namespace pfsp

extern "C" {

int pfsp_mlp_create(int m, uint64_t seed, pfsp_mlp **out) {
    if (!out) return set_error(PFSP_ERR_INVALID, "NULL argument");
    if (m < 2 || m > 20) return set_error(PFSP_ERR_UNSUPPORTED, "the ordering network supports 2 <= m <= 20");
    pfsp_mlp *M = (pfsp_mlp *)calloc(1, sizeof(pfsp_mlp));
    if (!M) return set_error(PFSP_ERR_OOM, "host allocation failed");
    M->m = m;
    M->P = m * (m - 1) / 2;
    M->D0 = round16(3 * m);
    M->H = kMlpHidden;
    M->O = round16(1 + M->P);
    cudaGetDevice(&M->device);
    size_t o = 0;
    M->oW1 = o; o += (size_t)M->D0 * M->H;
    M->ob1 = o; o += M->H;
    M->oW2 = o; o += (size_t)M->H * M->H;
    M->ob2 = o; o += M->H;
    M->oW3 = o; o += (size_t)M->H * M->O;
    M->ob3 = o; o += M->O;
    M->n_params = o;
    // He-uniform initialisation from a SplitMix64 stream; padded input rows
    // and padded output columns start (and, untrained, stay) at zero
    std::vector<float> h(o, 0.0f);
    uint64_t s = seed;
    auto uni = [&]() { return (double)(splitmix(s) >> 11) * (1.0 / 9007199254740992.0); };
    auto fill = [&](size_t off, int K, int N, int kreal, int nreal) {
        float a = (float)std::sqrt(6.0 / K);
        for (int k = 0; k < K; ++k)
            for (int nn = 0; nn < N; ++nn) {
                float v = (float)((2.0 * uni() - 1.0) * a);
                h[off + (size_t)k * N + nn] = (k < kreal && nn < nreal) ? v : 0.0f;
            }
    };
    fill(M->oW1, M->D0, M->H, 3 * m, M->H);
    fill(M->oW2, M->H, M->H, M->H, M->H);
    fill(M->oW3, M->H, M->O, M->H, 1 + M->P);
    size_t nb = o * sizeof(float);
    cudaError_t e = cudaMalloc(&M->params, nb);
    if (e == cudaSuccess) e = cudaMalloc(&M->grads, nb);
    if (e == cudaSuccess) e = cudaMalloc(&M->adam_m, nb);
    if (e == cudaSuccess) e = cudaMalloc(&M->adam_v, nb);
    if (e == cudaSuccess)
        e = cudaMalloc(&M->wb, ((size_t)M->D0 * M->H + (size_t)M->H * M->H + (size_t)M->H * M->O) * 2);
    if (e == cudaSuccess) e = cudaMemcpy(M->params, h.data(), nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(M->grads, 0, nb);
    if (e == cudaSuccess) e = cudaMemset(M->adam_m, 0, nb);
    if (e == cudaSuccess) e = cudaMemset(M->adam_v, 0, nb);
    if (e == cudaSuccess) e = refresh(M);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(M->params);
        cudaFree(M->grads);
        cudaFree(M->adam_m);
        cudaFree(M->adam_v);
        cudaFree(M->wb);
        free(M);
        return set_error(PFSP_ERR_CUDA, "pfsp_mlp_create: %s", cudaGetErrorString(e));
    }
    *out = M;
    return PFSP_OK;
}

void pfsp_mlp_free(pfsp_mlp *M) {
    if (!M) return;
    cudaFree(M->params);
    cudaFree(M->grads);
    cudaFree(M->adam_m);
    cudaFree(M->adam_v);
    cudaFree(M->wb);
    free(M);
}

int pfsp_mlp_shape(const pfsp_mlp *M, int *D0, int *H, int *O, int *P, int64_t *n_params) {
    if (!M) return set_error(PFSP_ERR_INVALID, "NULL argument");
    if (D0) *D0 = M->D0;
    if (H) *H = M->H;
    if (O) *O = M->O;
    if (P) *P = M->P;
    if (n_params) *n_params = (int64_t)M->n_params;
    return PFSP_OK;
}

int pfsp_mlp_get_params(const pfsp_mlp *M, float *out) {
    if (!M || !out) return set_error(PFSP_ERR_INVALID, "NULL argument");
    cudaError_t e = cudaMemcpy(out, M->params, M->n_params * 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? PFSP_OK : set_error(PFSP_ERR_CUDA, "%s", cudaGetErrorString(e));
}

int pfsp_mlp_set_params(pfsp_mlp *M, const float *in) {
    if (!M || !in) return set_error(PFSP_ERR_INVALID, "NULL argument");
    cudaError_t e = cudaMemcpy(M->params, in, M->n_params * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = refresh(M);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e == cudaSuccess ? PFSP_OK : set_error(PFSP_ERR_CUDA, "%s", cudaGetErrorString(e));
}

}  // extern "C"

namespace pfsp {

// Logits dY [rows][O] of device inputs dX [rows][D0] (synchronous): the
// tcgen05 kernel of mlp_tc.cu; cudaErrorTimeout when one of its bounded
// waits expired.
cudaError_t mlp_forward_dev(const pfsp_mlp *M, const float *dX, long long rows, float *dY) {
    bool timed_out = false;
    cudaError_t e = mlp_forward_tc(mlp_view(M), dX, rows, dY, 0, &timed_out);
    if (e == cudaSuccess && timed_out) e = cudaErrorTimeout;
    return e;
}

}  // namespace pfsp

extern "C" {

int pfsp_mlp_forward(const pfsp_mlp *M, int64_t rows, const float *X, float *Y) {
    if (!M || (rows > 0 && (!X || !Y)) || rows < 0) return set_error(PFSP_ERR_INVALID, "bad argument");
    if (rows == 0) return PFSP_OK;
    float *dX = nullptr, *dY = nullptr;
    cudaError_t e = cudaMalloc(&dX, rows * M->D0 * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dY, rows * M->O * 4);
    if (e == cudaSuccess) e = cudaMemcpy(dX, X, rows * M->D0 * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = pfsp::mlp_forward_dev(M, dX, rows, dY);
    if (e == cudaSuccess) e = cudaMemcpy(Y, dY, rows * M->O * 4, cudaMemcpyDeviceToHost);
    cudaFree(dX);
    cudaFree(dY);
    if (e == cudaErrorTimeout) return set_error(PFSP_ERR_TIMEOUT, "pfsp_mlp_forward: a bounded device wait expired");
    return e == cudaSuccess ? PFSP_OK : set_error(PFSP_ERR_CUDA, "pfsp_mlp_forward: %s", cudaGetErrorString(e));
}

// Loss and gradient (same layout as the parameters) of the masked mean BCE
// over all `rows`, without changing the parameters.
int pfsp_mlp_loss_grad(const pfsp_mlp *Mc, int64_t rows, const float *X, const float *T, const float *Mk,
                       float *loss, float *grad) {
    pfsp_mlp *M = const_cast<pfsp_mlp *>(Mc);
    if (!M || rows <= 0 || !X || !T || !Mk || !loss || !grad) return set_error(PFSP_ERR_INVALID, "bad argument");
    if (rows > (1 << 30)) return set_error(PFSP_ERR_UNSUPPORTED, "too many rows");
    float *dX = nullptr, *dT = nullptr, *dM = nullptr, *dl = nullptr;
    cudaError_t e = cudaMalloc(&dX, rows * M->D0 * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dT, rows * M->O * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dM, rows * M->O * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dl, 4);
    if (e == cudaSuccess) e = cudaMemcpy(dX, X, rows * M->D0 * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dT, T, rows * M->O * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dM, Mk, rows * M->O * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(dl, 0, 4);
    if (e == cudaSuccess) e = cudaMemset(M->grads, 0, M->n_params * 4);
    size_t smem = 0;
    int nsm = grad_blocks_and_smem(M, 4, &smem);
    if (e == cudaSuccess) {
        mlp_grad_kernel<<<nsm * 2, 128, smem>>>(mlp_view(M), dX, dT, dM, nullptr, 0, (int)rows, 1.0f / (float)rows,
                                                M->grads, M->oW1, M->ob1, M->oW2, M->ob2, M->oW3, M->ob3, dl);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(grad, M->grads, M->n_params * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(loss, dl, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(M->grads, 0, M->n_params * 4);
    cudaFree(dX);
    cudaFree(dT);
    cudaFree(dM);
    cudaFree(dl);
    return e == cudaSuccess ? PFSP_OK : set_error(PFSP_ERR_CUDA, "pfsp_mlp_loss_grad: %s", cudaGetErrorString(e));
}

// Train with Adam on mini-batches of a fixed permutation of the rows per
// epoch (SplitMix64-shuffled); epoch_loss (may be NULL) receives each
// epoch's mean loss.
int pfsp_mlp_train(pfsp_mlp *M, int64_t rows, const float *X, const float *T, const float *Mk, int epochs,
                   int batch, float lr, uint64_t seed, float *epoch_loss) {
    if (!M || rows <= 0 || !X || !T || !Mk || epochs < 1 || batch < 1 || lr <= 0)
        return set_error(PFSP_ERR_INVALID, "bad argument");
    if (rows > (1 << 30)) return set_error(PFSP_ERR_UNSUPPORTED, "too many rows");
    float *dX = nullptr, *dT = nullptr, *dM = nullptr, *dl = nullptr;
    int *didx = nullptr;
    cudaError_t e = cudaMalloc(&dX, rows * M->D0 * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dT, rows * M->O * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dM, rows * M->O * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dl, 4 * (size_t)epochs);
    if (e == cudaSuccess) e = cudaMalloc(&didx, rows * 4);
    if (e == cudaSuccess) e = cudaMemcpy(dX, X, rows * M->D0 * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dT, T, rows * M->O * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dM, Mk, rows * M->O * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(dl, 0, 4 * (size_t)epochs);
    if (e == cudaSuccess) e = cudaMemset(M->grads, 0, M->n_params * 4);
    size_t smem = 0;
    int nsm = grad_blocks_and_smem(M, 4, &smem);
    std::vector<int> perm(rows);
    uint64_t s = seed;
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
        for (int64_t i = 0; i < rows; ++i) perm[i] = (int)i;
        for (int64_t i = rows - 1; i > 0; --i) std::swap(perm[i], perm[splitmix(s) % (uint64_t)(i + 1)]);
        e = cudaMemcpy(didx, perm.data(), rows * 4, cudaMemcpyHostToDevice);
        for (int64_t b0 = 0; b0 < rows && e == cudaSuccess; b0 += batch) {
            int nb = (int)std::min<int64_t>(batch, rows - b0);
            int tiles = (nb + 15) / 16;
            int blocks = std::max(1, std::min(nsm * 2, (tiles + 3) / 4));
            mlp_grad_kernel<<<blocks, 128, smem>>>(mlp_view(M), dX, dT, dM, didx, b0, nb, 1.0f / (float)nb,
                                                   M->grads, M->oW1, M->ob1, M->oW2, M->ob2, M->oW3, M->ob3,
                                                   dl + ep);
            M->step += 1;
            const float b1 = 0.9f, b2 = 0.999f;
            float c1 = 1.0f - powf(b1, (float)M->step), c2 = 1.0f - powf(b2, (float)M->step);
            mlp_adam_kernel<<<64, 256>>>(M->params, M->grads, M->adam_m, M->adam_v, M->n_params, lr, b1, b2, 1e-8f,
                                         c1, c2);
            e = refresh(M);
        }
    }
    std::vector<float> hl(epochs);
    if (e == cudaSuccess) e = cudaMemcpy(hl.data(), dl, 4 * (size_t)epochs, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && epoch_loss) {
        int nbatches = (int)((rows + batch - 1) / batch);
        for (int ep = 0; ep < epochs; ++ep) epoch_loss[ep] = hl[ep] / nbatches;
    }
    cudaFree(dX);
    cudaFree(dT);
    cudaFree(dM);
    cudaFree(dl);
    cudaFree(didx);
    return e == cudaSuccess ? PFSP_OK : set_error(PFSP_ERR_CUDA, "pfsp_mlp_train: %s", cudaGetErrorString(e));
}

}  // extern "C"
