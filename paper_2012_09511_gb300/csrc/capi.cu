// capi.cu -- the library's C ABI: instance loading (with the host-built
// LB2 tables), batched bounding entry points, statistics and error messages.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "bound_device.cuh"
#include "pfsp_internal.h"

namespace pfsp {

static thread_local char g_err[512] = "";

int set_error(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

TableLayout table_layout(int n, int m) {
    TableLayout L;
    L.n = n;
    L.m = m;
    L.P = m * (m - 1) / 2;
    L.S = (L.P + 31) / 32;
    L.Ssweep = L.S;
    L.nj = (n + 3) & ~3;
    L.off_pm = 0;
    L.off_tot = L.off_pm + m * L.nj;
    L.off_pq = L.off_tot + 32;
    L.off_kl = L.off_pq + ((2 * n * m + 3) & ~3);
    L.off_rank = L.off_kl + L.S * 32;
    L.off_ptab = L.off_rank + L.S * n * 8;
    L.words = L.off_ptab + 2 * L.S * n * 32;
    return L;
}

// Johnson's rule extended to time lags (Mitten) for the pair (k, l): jobs
// with p_jk <= p_jl first by ascending p_jk + g_j, then the rest by
// descending p_jl + g_j; ties by ascending job id (Section 2.4, LB2).
static std::vector<int> johnson_lag_order(int n, int m, const int32_t *p, int k, int l,
                                          const std::vector<int> &lag) {
    std::vector<int> ord(n);
    std::iota(ord.begin(), ord.end(), 0);
    auto first = [&](int j) { return p[j * m + k] <= p[j * m + l]; };
    std::sort(ord.begin(), ord.end(), [&](int x, int y) {
        bool fx = first(x), fy = first(y);
        if (fx != fy) return fx;
        if (fx) {
            int kx = p[x * m + k] + lag[x], ky = p[y * m + k] + lag[y];
            if (kx != ky) return kx < ky;
        } else {
            int kx = p[x * m + l] + lag[x], ky = p[y * m + l] + lag[y];
            if (kx != ky) return kx > ky;
        }
        return x < y;
    });
    return ord;
}

void build_tables(const TableLayout &L, const int32_t *p, std::vector<int32_t> &blob, const int32_t *pair_order,
                  int count) {
    const int n = L.n, m = L.m;
    // slot position of every pair: pair_order[i] = the pair at position i;
    // pairs beyond the first `count` positions are left out (-1)
    std::vector<int> where(L.P, -1);
    for (int i = 0; i < count; ++i) where[pair_order ? pair_order[i] : i] = i;
    blob.assign(L.words, 0);
    for (int k = 0; k < m; ++k)
        for (int j = 0; j < n; ++j) blob[L.off_pm + k * L.nj + j] = p[j * m + k];
    for (int k = 0; k < m; ++k) {
        int32_t t = 0;
        for (int j = 0; j < n; ++j) t += p[j * m + k];
        blob[L.off_tot + k] = t;
    }
    for (int j = 0; j < n; ++j) {
        int32_t pre = 0, suf = 0;
        for (int k = 0; k < m; ++k) {
            pre += p[j * m + k];
            suf += p[j * m + (m - 1 - k)];
            blob[L.off_pq + 2 * (j * m + k)] = pre;                // P_k
            blob[L.off_pq + 2 * (j * m + (m - 1 - k)) + 1] = suf;  // Q_{m-1-k}
        }
    }
    // bit of position t in the kernels' position masks: 31 - t for n <= 32, t above
    auto pos_bit = [n](int t) { return n <= 32 ? 31 - t : t; };
    int2 *ptab = reinterpret_cast<int2 *>(blob.data() + L.off_ptab);
    uint8_t *rank = reinterpret_cast<uint8_t *>(blob.data() + L.off_rank);
    for (int s = 0; s < L.S; ++s)
        for (int t = 0; t < n; ++t)
            for (int lane = 0; lane < 32; ++lane) {
                ptab[(s * n + t) * 32 + lane] = make_int2(t, kNegInf);
                rank[(t * L.S + s) * 32 + lane] = (uint8_t)pos_bit(t);
            }
    int q = 0;
    std::vector<int> lag(n);
    for (int k = 0; k < m; ++k)
        for (int l = k + 1; l < m; ++l, ++q) {
            if (where[q] < 0) continue;
            const int s = where[q] / 32, lane = where[q] % 32;
            blob[L.off_kl + where[q]] = k | (l << 8);
            for (int j = 0; j < n; ++j) {
                int g = 0;
                for (int r = k + 1; r < l; ++r) g += p[j * m + r];
                lag[j] = g;
            }
            std::vector<int> ord = johnson_lag_order(n, m, p, k, l, lag);
            for (int t = 0; t < n; ++t) {
                int j = ord[t];
                int a = p[j * m + l] - p[j * m + k];
                int b = lag[j] + p[j * m + l];
                ptab[(s * n + t) * 32 + lane] = make_int2((int)((unsigned)a << 8) | j, b);
                rank[(j * L.S + s) * 32 + lane] = (uint8_t)pos_bit(t);
            }
        }
}

static int cuda_fail(cudaError_t e, const char *what) {
    return set_error(PFSP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

static int ensure_scratch(pfsp_instance *inst, size_t bytes) {
    if (inst->scratch_bytes >= bytes) return PFSP_OK;
    if (inst->d_scratch) cudaFree(inst->d_scratch);
    inst->d_scratch = nullptr;
    inst->scratch_bytes = 0;
    cudaError_t e = cudaMalloc(&inst->d_scratch, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(PFSP_ERR_OOM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    }
    inst->scratch_bytes = bytes;
    return PFSP_OK;
}

// The bounding kernel of the kind: with PFSP_MINHT the refined one.
static cudaError_t launch_bounds(const pfsp_instance *inst, int kind, long long num_nodes, const uint8_t *perm,
                                 const uint8_t *d1, const uint8_t *d2, int32_t *lb1, int32_t *lb2,
                                 cudaStream_t stream) {
    if (kind & PFSP_MINHT)
        return launch_bound_batch_minht(inst, kind & ~PFSP_MINHT, num_nodes, perm, d1, d2, lb1, lb2, stream);
    return launch_bound_batch(inst, kind, num_nodes, perm, d1, d2, lb1, lb2, stream);
}

static int check_bound_args(const pfsp_instance *inst, int kind, int64_t num_nodes, const void *perm,
                            const void *d1, const void *d2, const void *lb1, const void *lb2) {
    if (!inst) return set_error(PFSP_ERR_INVALID, "instance is NULL");
    if ((kind & (PFSP_LB1 | PFSP_LB2)) == 0 || (kind & ~(PFSP_LB1 | PFSP_LB2 | PFSP_MINHT)) != 0)
        return set_error(PFSP_ERR_INVALID, "kind must be a non-empty mask of LB1|LB2, optionally with PFSP_MINHT");
    if (num_nodes < 0) return set_error(PFSP_ERR_INVALID, "num_nodes < 0");
    if (num_nodes == 0) return PFSP_OK;
    if (!perm || !d1 || !d2) return set_error(PFSP_ERR_INVALID, "NULL node input");
    if ((kind & PFSP_LB1) && !lb1) return set_error(PFSP_ERR_INVALID, "LB1 requested but lb1_out is NULL");
    if ((kind & PFSP_LB2) && !lb2) return set_error(PFSP_ERR_INVALID, "LB2 requested but lb2_out is NULL");
    if ((kind & PFSP_LB2) && !inst->lb2_ok)
        return set_error(PFSP_ERR_UNSUPPORTED, "LB2 tables of %d pairs x %d jobs exceed shared memory",
                         inst->lay.P, inst->n);
    return PFSP_OK;
}

}  // namespace pfsp

using namespace pfsp;

extern "C" {

const char *pfsp_last_error(void) { return g_err; }

int pfsp_load_instance(int n, int m, const int32_t *p, pfsp_instance **out) {
    g_err[0] = 0;
    if (!p || !out) return set_error(PFSP_ERR_INVALID, "NULL argument");
    if (n < 1 || m < 1) return set_error(PFSP_ERR_INVALID, "n and m must be >= 1 (n=%d, m=%d)", n, m);
    if (n > kMaxJobs || m > kMaxMachines)
        return set_error(PFSP_ERR_UNSUPPORTED, "n <= %d and m <= %d required (n=%d, m=%d)", kMaxJobs,
                         kMaxMachines, n, m);
    long long total = 0;
    for (long long i = 0; i < (long long)n * m; ++i) {
        if (p[i] < 0) return set_error(PFSP_ERR_INVALID, "negative processing time at index %lld", i);
        if (p[i] > kMaxTime) return set_error(PFSP_ERR_UNSUPPORTED, "processing time above 2^22-1 at %lld", i);
        total += p[i];
    }
    if (total >= kMaxTotal) return set_error(PFSP_ERR_UNSUPPORTED, "sum of processing times >= 2^28");

    pfsp_instance *inst = (pfsp_instance *)calloc(1, sizeof(pfsp_instance));
    if (!inst) return set_error(PFSP_ERR_OOM, "host allocation failed");
    inst->n = n;
    inst->m = m;
    cudaGetDevice(&inst->device);
    inst->p_host = (int32_t *)malloc(sizeof(int32_t) * n * m);
    if (!inst->p_host) {
        free(inst);
        return set_error(PFSP_ERR_OOM, "host allocation failed");
    }
    memcpy(inst->p_host, p, sizeof(int32_t) * n * m);
    inst->lay = table_layout(n, m);
    // the limit counts the LB2 tables proper (the prefix/suffix sums add about 2 n m words)
    inst->lb2_ok = (size_t)(inst->lay.words - (inst->lay.off_kl - inst->lay.off_pq)) * 4 <= (size_t)kMaxTableBytes;
    std::vector<int32_t> blob;
    build_tables(inst->lay, p, blob, nullptr, inst->lay.P);
    cudaError_t e = cudaMalloc(&inst->d_tab, blob.size() * sizeof(int32_t));
    if (e != cudaSuccess) {
        cudaGetLastError();
        free(inst->p_host);
        free(inst);
        return set_error(PFSP_ERR_OOM, "cudaMalloc of instance tables failed: %s", cudaGetErrorString(e));
    }
    e = cudaMemcpy(inst->d_tab, blob.data(), blob.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(inst->d_tab);
        free(inst->p_host);
        free(inst);
        return cuda_fail(e, "upload of instance tables");
    }
    *out = inst;
    return PFSP_OK;
}

void pfsp_free_instance(pfsp_instance *inst) {
    if (!inst) return;
    if (inst->d_tab) cudaFree(inst->d_tab);
    if (inst->d_scratch) cudaFree(inst->d_scratch);
    free(inst->p_host);
    free(inst->pair_order);
    free(inst);
}

int pfsp_set_lb2_pairs(pfsp_instance *inst, const int32_t *pairs, int count) {
    g_err[0] = 0;
    if (!inst) return set_error(PFSP_ERR_INVALID, "instance is NULL");
    const int P = inst->lay.P;
    if (P == 0) return set_error(PFSP_ERR_INVALID, "an instance with one machine has no machine pair");
    if (pairs && (count < 1 || count > P)) return set_error(PFSP_ERR_INVALID, "count must be in 1..%d", P);
    if (!pairs) {
        // already every pair in index order: nothing to rebuild
        bool identity = inst->pair_count == 0 || inst->pair_count == P;
        for (int q = 0; identity && inst->pair_order && q < P; ++q) identity = inst->pair_order[q] == q;
        if (identity) return PFSP_OK;
        count = P;
    }
    std::vector<int32_t> ord(P);
    std::vector<char> seen(P, 0);
    int k = 0;
    if (pairs) {
        for (int i = 0; i < count; ++i) {
            if (pairs[i] < 0 || pairs[i] >= P || seen[pairs[i]])
                return set_error(PFSP_ERR_INVALID, "pairs must be distinct indices in 0..%d (entry %d)", P - 1, i);
            seen[pairs[i]] = 1;
            ord[k++] = pairs[i];
        }
    }
    for (int q = 0; q < P; ++q)
        if (!seen[q]) ord[k++] = q;  // the pairs left out, after the ones in use
    std::vector<int32_t> blob;
    build_tables(inst->lay, inst->p_host, blob, ord.data(), count);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMemcpy(inst->d_tab, blob.data(), blob.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "upload of the instance tables");
    if (!inst->pair_order) inst->pair_order = (int32_t *)malloc(sizeof(int32_t) * P);
    if (!inst->pair_order) return set_error(PFSP_ERR_OOM, "host allocation failed");
    memcpy(inst->pair_order, ord.data(), sizeof(int32_t) * P);
    inst->pair_count = count;
    inst->lay.Ssweep = (count + 31) / 32;
    return PFSP_OK;
}

int pfsp_set_pair_order(pfsp_instance *inst, const int32_t *order) {
    g_err[0] = 0;
    if (!inst) return set_error(PFSP_ERR_INVALID, "instance is NULL");
    const int P = inst->lay.P;
    if (order) {
        std::vector<char> seen(P, 0);
        for (int i = 0; i < P; ++i) {
            if (order[i] < 0 || order[i] >= P || seen[order[i]])
                return set_error(PFSP_ERR_INVALID, "order is not a permutation of 0..%d (entry %d)", P - 1, i);
            seen[order[i]] = 1;
        }
    }
    if (P == 0) return PFSP_OK;
    return pfsp_set_lb2_pairs(inst, order, P);
}

int pfsp_get_pair_order(const pfsp_instance *inst, int32_t *order) {
    g_err[0] = 0;
    if (!inst || !order) return set_error(PFSP_ERR_INVALID, "NULL argument");
    const int used = inst->pair_count > 0 ? inst->pair_count : inst->lay.P;
    for (int i = 0; i < inst->lay.P; ++i)
        order[i] = i < used ? (inst->pair_order ? inst->pair_order[i] : i) : -1;
    return PFSP_OK;
}

int pfsp_bound_batch_dev(const pfsp_instance *inst, int kind, int64_t num_nodes, const uint8_t *perm,
                         const uint8_t *d1, const uint8_t *d2, int32_t *lb1_out, int32_t *lb2_out, void *stream) {
    g_err[0] = 0;
    int rc = check_bound_args(inst, kind, num_nodes, perm, d1, d2, lb1_out, lb2_out);
    if (rc != PFSP_OK || num_nodes == 0) return rc;
    cudaError_t e = launch_bounds(inst, kind, num_nodes, perm, d1, d2, (kind & PFSP_LB1) ? lb1_out : nullptr,
                                       (kind & PFSP_LB2) ? lb2_out : nullptr, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "bound kernel launch");
    return PFSP_OK;
}

// The device address of host buffer [h, h + bytes) when all of it is
// page-locked memory that the current device maps as one contiguous range
// (both ends checked), else NULL: pageable memory, or a range the checks
// cannot vouch for, is never handed to a kernel.
static char *mapped_host(void *h, size_t bytes) {
    if (!h || bytes == 0) return nullptr;
    int dev = 0, can_map = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&can_map, cudaDevAttrCanMapHostMemory, dev) != cudaSuccess || !can_map) {
        cudaGetLastError();
        return nullptr;
    }
    cudaPointerAttributes a0, a1;
    if (cudaPointerGetAttributes(&a0, h) != cudaSuccess ||
        cudaPointerGetAttributes(&a1, (const char *)h + (bytes - 1)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a0.type != cudaMemoryTypeHost || a1.type != cudaMemoryTypeHost || !a0.devicePointer || !a1.devicePointer)
        return nullptr;
    if ((char *)a1.devicePointer != (char *)a0.devicePointer + (bytes - 1)) return nullptr;
    return (char *)a0.devicePointer;
}

// Host-pointer bounding, shared by both modes: the bound arrays (summary
// NULL) or one summary per node (reduce mode, survivors below ub).
static int bound_host(pfsp_instance *inst, int kind, int64_t num_nodes, const uint8_t *perm, const uint8_t *d1,
                      const uint8_t *d2, int32_t *lb1_out, int32_t *lb2_out, pfsp_node_summary *summary, int ub) {
    auto t0 = std::chrono::steady_clock::now();
    const int n = inst->n;
    if (num_nodes == 0) return PFSP_OK;
    // Chunks of the batch alternate between two streams, so that the copies
    // of one chunk (nodes in, both bound arrays out) overlap the kernel of the
    // other; each stream reuses its own device buffers in stream order.
    const int64_t chunk = std::min<int64_t>(num_nodes, kBoundChunk);
    const int64_t nchunks = (num_nodes + chunk - 1) / chunk;
    const int nst = nchunks > 1 ? 2 : 1;
    const size_t in_bytes = (size_t)chunk * (n + 2);
    const size_t out_bytes = summary ? (size_t)chunk * sizeof(pfsp_node_summary) : (size_t)chunk * 2 * n * sizeof(int32_t);
    const bool want1 = !summary && (kind & PFSP_LB1), want2 = !summary && (kind & PFSP_LB2);
    const size_t off_out1 = (in_bytes + 255) & ~(size_t)255;
    const size_t off_out2 = off_out1 + (((want1 || summary) ? out_bytes : 0) + 255) / 256 * 256;
    const size_t per_stream = (off_out2 + (want2 ? out_bytes : 0) + 255) / 256 * 256;
    int rc = ensure_scratch(inst, per_stream * nst);
    if (rc != PFSP_OK) return rc;
    // The chunks after the first nst write their results straight into the
    // caller's buffers when those are page-locked host memory that the GPU
    // maps: the kernel's stores cross the host link while it runs, so no copy
    // is left to wait for after the last kernel.  Pageable buffers, and the
    // first chunks (whose results wait for the host's validation of the
    // depths), go through device buffers and copies.
    const size_t row_bytes = (size_t)2 * n * sizeof(int32_t);
    char *z1 = want1 ? mapped_host(lb1_out, (size_t)num_nodes * row_bytes) : nullptr;
    char *z2 = want2 ? mapped_host(lb2_out, (size_t)num_nodes * row_bytes) : nullptr;
    char *zs = summary ? mapped_host(summary, (size_t)num_nodes * sizeof(pfsp_node_summary)) : nullptr;
    const bool direct = nchunks > nst && (!want1 || z1) && (!want2 || z2) && (!summary || zs);
    cudaStream_t st[2] = {nullptr, nullptr};
    std::vector<cudaEvent_t> evs((size_t)nchunks * 2, nullptr);
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < nst && e == cudaSuccess; ++q) e = cudaStreamCreateWithFlags(&st[q], cudaStreamNonBlocking);
    for (size_t q = 0; q < evs.size() && e == cudaSuccess; ++q) e = cudaEventCreate(&evs[q]);
    struct Bufs {
        uint8_t *perm, *d1, *d2;
        int32_t *o1, *o2;
        pfsp_node_summary *os;
    };
    auto bufs = [&](int64_t c) {
        char *base = (char *)inst->d_scratch + per_stream * (size_t)(c % nst);
        const int64_t cn = std::min<int64_t>(chunk, num_nodes - c * chunk);
        Bufs b;
        b.perm = (uint8_t *)base;
        b.d1 = b.perm + (size_t)cn * n;
        b.d2 = b.d1 + cn;
        b.o1 = want1 ? (int32_t *)(base + off_out1) : nullptr;
        b.o2 = want2 ? (int32_t *)(base + off_out2) : nullptr;
        b.os = summary ? (pfsp_node_summary *)(base + off_out1) : nullptr;
        return b;
    };
    // nodes in and the kernel of chunk c
    auto front = [&](int64_t c) {
        const int q = (int)(c % nst);
        const int64_t off = c * chunk, cn = std::min<int64_t>(chunk, num_nodes - off);
        Bufs b = bufs(c);
        if (direct && c >= nst) {
            b.o1 = want1 ? (int32_t *)(z1 + (size_t)off * row_bytes) : nullptr;
            b.o2 = want2 ? (int32_t *)(z2 + (size_t)off * row_bytes) : nullptr;
            b.os = summary ? (pfsp_node_summary *)(zs + (size_t)off * sizeof(pfsp_node_summary)) : nullptr;
        }
        cudaError_t r = cudaMemcpyAsync(b.perm, perm + (size_t)off * n, (size_t)cn * n, cudaMemcpyHostToDevice, st[q]);
        if (r == cudaSuccess) r = cudaMemcpyAsync(b.d1, d1 + off, cn, cudaMemcpyHostToDevice, st[q]);
        if (r == cudaSuccess) r = cudaMemcpyAsync(b.d2, d2 + off, cn, cudaMemcpyHostToDevice, st[q]);
        if (r == cudaSuccess) r = cudaEventRecord(evs[2 * c], st[q]);
        if (r == cudaSuccess)
            r = summary ? launch_bound_batch(inst, kind, cn, b.perm, b.d1, b.d2, nullptr, nullptr, st[q], b.os, ub)
                        : launch_bounds(inst, kind, cn, b.perm, b.d1, b.d2, b.o1, b.o2, st[q]);
        if (r == cudaSuccess) r = cudaEventRecord(evs[2 * c + 1], st[q]);
        return r;
    };
    // the results of chunk c back to the caller's buffers
    auto back = [&](int64_t c) {
        if (direct && c >= nst) return cudaSuccess;  // written in place by the kernel
        const int q = (int)(c % nst);
        const int64_t off = c * chunk, cn = std::min<int64_t>(chunk, num_nodes - off);
        const Bufs b = bufs(c);
        const size_t ob = (size_t)cn * 2 * n * sizeof(int32_t);
        cudaError_t r = cudaSuccess;
        if (b.os)
            r = cudaMemcpyAsync(summary + off, b.os, (size_t)cn * sizeof(pfsp_node_summary), cudaMemcpyDeviceToHost,
                                st[q]);
        if (r == cudaSuccess && b.o1) r = cudaMemcpyAsync(lb1_out + (size_t)off * 2 * n, b.o1, ob, cudaMemcpyDeviceToHost, st[q]);
        if (r == cudaSuccess && b.o2) r = cudaMemcpyAsync(lb2_out + (size_t)off * 2 * n, b.o2, ob, cudaMemcpyDeviceToHost, st[q]);
        return r;
    };
    // The first chunk of each stream goes in before the host validates the
    // depths, so that the validation overlaps their copies and kernels; no
    // result is copied back before it passes, so a rejected batch leaves the
    // caller's buffers untouched (the kernel itself writes -1 for a node with
    // d1 + d2 > n and reads nothing past its row).
    for (int64_t c = 0; c < nst && e == cudaSuccess; ++c) e = front(c);
    // one pass over the depths: validation and the children count (a plain
    // reduction the host compiler vectorises)
    uint64_t depth_sum = 0;
    unsigned dmax = 0;
    for (int64_t i0 = 0; i0 < num_nodes; i0 += 1 << 16) {
        const int64_t i1 = std::min<int64_t>(num_nodes, i0 + (1 << 16));
        uint32_t part = 0;  // at most 65,536 x 128: no overflow
        for (int64_t i = i0; i < i1; ++i) {
            const unsigned d = (unsigned)d1[i] + (unsigned)d2[i];
            part += d;
            dmax = d > dmax ? d : dmax;
        }
        depth_sum += part;
    }
    if (dmax > (unsigned)n) {
        for (int64_t i = 0; i < num_nodes; ++i)
            if ((int)d1[i] + (int)d2[i] > n) {
                rc = set_error(PFSP_ERR_INVALID, "node %lld: d1 + d2 = %d > n = %d", (long long)i, d1[i] + d2[i], n);
                break;
            }
    }
    if (rc == PFSP_OK) {
        for (int64_t c = 0; c < nchunks && e == cudaSuccess; ++c) {
            if (c >= nst) e = front(c);  // after back(c - nst): the stream's buffers are free again
            if (e == cudaSuccess) e = back(c);
        }
    }
    for (int q = 0; q < nst; ++q)
        if (st[q]) {
            cudaError_t e2 = cudaStreamSynchronize(st[q]);
            if (e == cudaSuccess) e = e2;
        }
    float ms = 0.f;
    for (int64_t c = 0; c < nchunks && e == cudaSuccess && rc == PFSP_OK; ++c) {
        float t = 0.f;
        e = cudaEventElapsedTime(&t, evs[2 * c], evs[2 * c + 1]);
        ms += t;
    }
    for (cudaEvent_t ev : evs)
        if (ev) cudaEventDestroy(ev);
    for (int q = 0; q < nst; ++q)
        if (st[q]) cudaStreamDestroy(st[q]);
    if (e != cudaSuccess) return cuda_fail(e, summary ? "pfsp_bound_reduce" : "pfsp_bound_batch");
    if (rc != PFSP_OK) return rc;
    memset(&inst->stats, 0, sizeof(inst->stats));
    const uint64_t children = 2 * ((uint64_t)num_nodes * (uint64_t)n - depth_sum);
    inst->stats.decomposed = (uint64_t)num_nodes;
    inst->stats.bounded_children = children;
    inst->stats.kernel_seconds = ms * 1e-3;
    inst->stats.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return PFSP_OK;
}

int pfsp_bound_batch(const pfsp_instance *inst_c, int kind, int64_t num_nodes, const uint8_t *perm,
                     const uint8_t *d1, const uint8_t *d2, int32_t *lb1_out, int32_t *lb2_out) {
    g_err[0] = 0;
    pfsp_instance *inst = const_cast<pfsp_instance *>(inst_c);
    int rc = check_bound_args(inst, kind, num_nodes, perm, d1, d2, lb1_out, lb2_out);
    if (rc != PFSP_OK) return rc;
    return bound_host(inst, kind, num_nodes, perm, d1, d2, lb1_out, lb2_out, nullptr, 0);
}

static int check_reduce_args(const pfsp_instance *inst, int kind, int64_t num_nodes, const void *perm,
                             const void *d1, const void *d2, const void *out) {
    if (kind != PFSP_LB1 && kind != PFSP_LB2) return set_error(PFSP_ERR_INVALID, "kind must be PFSP_LB1 or PFSP_LB2");
    int rc = check_bound_args(inst, kind, num_nodes, perm, d1, d2, out, out);
    if (rc != PFSP_OK) return rc;
    if (num_nodes > 0 && !out) return set_error(PFSP_ERR_INVALID, "out is NULL");
    return PFSP_OK;
}

int pfsp_bound_reduce(const pfsp_instance *inst_c, int kind, int64_t num_nodes, const uint8_t *perm,
                      const uint8_t *d1, const uint8_t *d2, int32_t ub, pfsp_node_summary *out) {
    g_err[0] = 0;
    pfsp_instance *inst = const_cast<pfsp_instance *>(inst_c);
    int rc = check_reduce_args(inst, kind, num_nodes, perm, d1, d2, out);
    if (rc != PFSP_OK) return rc;
    return bound_host(inst, kind, num_nodes, perm, d1, d2, nullptr, nullptr, out, ub);
}

int pfsp_bound_reduce_dev(const pfsp_instance *inst, int kind, int64_t num_nodes, const uint8_t *perm,
                          const uint8_t *d1, const uint8_t *d2, int32_t ub, pfsp_node_summary *out, void *stream) {
    g_err[0] = 0;
    int rc = check_reduce_args(inst, kind, num_nodes, perm, d1, d2, out);
    if (rc != PFSP_OK || num_nodes == 0) return rc;
    cudaError_t e = launch_bound_batch(inst, kind, num_nodes, perm, d1, d2, nullptr, nullptr, (cudaStream_t)stream,
                                       out, ub);
    if (e != cudaSuccess) return cuda_fail(e, "bound kernel launch");
    return PFSP_OK;
}

int pfsp_stats(const pfsp_instance *inst, pfsp_stats_t *out) {
    if (!inst || !out) return set_error(PFSP_ERR_INVALID, "NULL argument");
    *out = inst->stats;
    return PFSP_OK;
}

}  // extern "C"
