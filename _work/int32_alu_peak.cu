// int32_alu_peak.cu -- INT32 throughput per SM per clock on this GPU, the
// denominator of the bounding kernel's ALU roofline.  Each thread runs eight
// independent chains of one instruction kind; cycles come from clock64() so
// the figure does not depend on the clock the GPU ran at.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o int32_alu_peak int32_alu_peak.cu
#include <cstdio>
#include <cuda_runtime.h>

#define ILP 8
template <int KIND>
__global__ void chains(int iters, int b, int c, int *out, long long *cyc) {
    int a[ILP];
#pragma unroll
    for (int i = 0; i < ILP; ++i) a[i] = threadIdx.x + i;
    __syncthreads();
    long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < ILP; ++i) {
            if (KIND == 0) asm volatile("max.s32 %0, %0, %1;" : "+r"(a[i]) : "r"(b));
            if (KIND == 1) asm volatile("add.s32 %0, %0, %1;" : "+r"(a[i]) : "r"(b));
            if (KIND == 2) a[i] = __viaddmax_s32(a[i], b, c);
            if (KIND == 3) asm volatile("mad.lo.s32 %0, %0, %1, %2;" : "+r"(a[i]) : "r"(b), "r"(c));
        }
    }
    __syncthreads();
    long long t1 = clock64();
    int s = 0;
#pragma unroll
    for (int i = 0; i < ILP; ++i) s += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

template <int KIND>
static void run(const char *name, int nsm) {
    const int threads = 1024, blocks = nsm, iters = 20000;
    int *out;
    long long *cyc;
    cudaMalloc(&out, sizeof(int) * threads * blocks);
    cudaMalloc(&cyc, sizeof(long long) * blocks);
    chains<KIND><<<blocks, threads>>>(100, 3, 5, out, cyc);
    chains<KIND><<<blocks, threads>>>(iters, 3, 5, out, cyc);
    cudaDeviceSynchronize();
    long long *h = new long long[blocks];
    cudaMemcpy(h, cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost);
    double avg = 0;
    for (int i = 0; i < blocks; ++i) avg += h[i];
    avg /= blocks;
    printf("%-9s thread-instructions per SM per clock = %.1f\n", name, (double)threads * iters * ILP / avg);
    cudaFree(out);
    cudaFree(cyc);
    delete[] h;
}

int main() {
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
    printf("SMs %d\n", nsm);
    run<0>("imax", nsm);
    run<1>("iadd", nsm);  // the compiler may fuse two adds into one IADD3
    run<2>("viaddmax", nsm);
    run<3>("imad", nsm);
    return 0;
}
