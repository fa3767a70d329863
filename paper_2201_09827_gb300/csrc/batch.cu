// Batches of independent systems and the autotuner that picks their launch shapes.
//
// gir_batch_solve runs Algorithm 4 on every system of a batch. Where the persistent kernel
// (k_persist.cu) implements the parameters, the whole batch is one launch of it. Otherwise the
// systems, which are independent (no exchange step), are scheduled longest-first (by n, the LU is
// O(n^3)) onto a pool of worker threads, each driving its own CUDA stream: small systems that
// cannot fill the GPU alone run side by side. The pool size and the LU outer block width of each size class come
// from a process-wide table filled by gir_autotune, which times the candidates on synthetic
// matrices of the class; classes without a measurement use the defaults (256, 8 workers).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "gir_batch.cuh"
#include "gir_internal.cuh"
#include "gir_persist.cuh"

namespace gir {
namespace {

struct ClassEntry {
    int64_t n_max = 0;  // largest order measured for the class
    int nb = 0;
    float ms = 0.0f;
};

std::mutex g_tune_mu;
std::map<int, ClassEntry> g_classes;  // size class c: n in (2^(c-1), 2^c]
int g_workers = 0;                    // 0: not measured

int size_class(int64_t n) {
    int c = 0;
    while (((int64_t)1 << c) < n) ++c;
    return c;
}

// Uniform entries in [-1, 1) from a 64-bit hash of the index (a synthetic tuning input).
__global__ void k_fill_hash(double* A, int64_t count, unsigned long long seed) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long z = (unsigned long long)i * 0x9E3779B97F4A7C15ull + seed;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        A[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    }
}

gir_params tuning_params(int nb) {
    gir_params p;
    memset(&p, 0, sizeof(p));
    p.uf = GIR_BF16;
    p.u = GIR_FP64;
    p.ur = GIR_FP64;
    p.ua = GIR_FP64;
    p.m = 30;
    p.k = 8;
    p.tau = 1e-8;
    p.imax = 10;
    p.target_berr = -1.0;
    p.carry_mode = 1;
    p.lu_nb = nb;
    return p;
}

// Device time of one gir_factor of A (order n) with outer block nb (best of reps), or < 0.
float time_factor(const double* A, int64_t n, int nb, int reps, cudaStream_t s) {
    gir_params p = tuning_params(nb);
    float best = -1.0f;
    for (int r = 0; r < reps + 1; ++r) {
        gir_handle* h = nullptr;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, s);
        gir_status st = gir_factor(A, n, n, &p, s, &h);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (h) {
            cudaStreamSynchronize(s);
            release_handle_on(h, s);
        }
        if (st != GIR_OK) return -1.0f;
        if (r > 0 && (best < 0.0f || ms < best)) best = ms;  // the first run warms up
    }
    return best;
}

// Wall time of factoring `count` synthetic systems of order n with `workers` concurrent streams.
float time_pool(const double* A, int64_t n, int count, int workers, int nb) {
    std::atomic<int> next{0};
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceSynchronize();
    auto t0 = std::chrono::steady_clock::now();
    std::vector<std::thread> th;
    std::atomic<int> failed{0};
    for (int w = 0; w < workers; ++w) {
        th.emplace_back([&, w]() {
            (void)w;
            cudaSetDevice(dev);
            cudaStream_t s;
            cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
            gir_params p = tuning_params(nb);
            for (int i = next++; i < count; i = next++) {
                gir_handle* h = nullptr;
                if (gir_factor(A, n, n, &p, s, &h) != GIR_OK) failed++;
                if (h) {
                    cudaStreamSynchronize(s);
                    release_handle_on(h, s);
                }
            }
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        });
    }
    for (auto& t : th) t.join();
    auto t1 = std::chrono::steady_clock::now();
    if (failed) return -1.0f;
    return std::chrono::duration<float, std::milli>(t1 - t0).count();
}

}  // namespace

int tuned_lu_nb(int64_t n) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_classes.find(size_class(n));
    return it == g_classes.end() ? 0 : it->second.nb;
}

}  // namespace gir

using namespace gir;

extern "C" {

gir_status gir_autotune(const int64_t* n, int count, void* stream) {
    if (count < 0 || (count > 0 && !n)) return GIR_INVALID_ARG;
    for (int i = 0; i < count; ++i)
        if (n[i] < 1) return GIR_INVALID_ARG;
    if (count == 0) return GIR_OK;
    cudaStream_t s = (cudaStream_t)stream;
    // classes to measure and their largest orders
    std::map<int, int64_t> todo;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (int i = 0; i < count; ++i) {
            const int c = size_class(n[i]);
            if (g_classes.count(c)) continue;
            todo[c] = std::max<int64_t>(todo[c], n[i]);
        }
    }
    int64_t nmax = 0;
    for (auto& kv : todo) nmax = std::max(nmax, kv.second);
    std::vector<int64_t> sorted(n, n + count);
    std::sort(sorted.begin(), sorted.end());
    const int64_t nmed = sorted[count / 2];
    const bool tune_workers = (g_workers == 0) && count > 1;
    if (tune_workers) nmax = std::max(nmax, nmed);
    if (nmax == 0) return GIR_OK;
    double* A = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void**>(&A), (size_t)nmax * nmax * sizeof(double), s) != cudaSuccess) {
        cudaGetLastError();
        return GIR_OOM;
    }
    count_launch(), k_fill_hash<<<1024, 256, 0, s>>>(A, nmax * nmax, 0x5eedull);
    cudaStreamSynchronize(s);
    gir_status st = GIR_OK;
    // A (order nmax, row-major) doubles as an order-m matrix with leading dimension m for m <= nmax
    for (auto& kv : todo) {
        const int64_t m = kv.second;
        ClassEntry best;
        best.n_max = m;
        const int cands[] = {64, 128, 256};
        for (int nb : cands) {
            if (nb > 64 && nb >= 2 * m) continue;   // wider than two blocks of the matrix: same as smaller
            const float ms = time_factor(A, m, nb, 2, s);
            if (ms >= 0.0f && (best.nb == 0 || ms < best.ms)) {
                best.nb = nb;
                best.ms = ms;
            }
        }
        if (best.nb == 0) {
            st = GIR_CUDA_ERROR;
            break;
        }
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_classes[kv.first] = best;
    }
    if (st == GIR_OK && tune_workers) {
        const int nb = tuned_lu_nb(nmed);
        const int batch = 32;
        int best_w = 0;
        float best_ms = 0.0f;
        for (int w : {2, 4, 8, 16}) {
            const float ms = time_pool(A, nmed, batch, w, nb);
            if (ms >= 0.0f && (best_w == 0 || ms < best_ms)) {
                best_w = w;
                best_ms = ms;
            }
        }
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_workers = best_w > 0 ? best_w : 8;
    }
    cudaFreeAsync(A, s);
    cudaStreamSynchronize(s);
    return st;
}

int gir_tune_report(char* buf, int buflen) {
    std::string out;
    char line[160];
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (auto& kv : g_classes) {
            snprintf(line, sizeof(line), "class %d: n <= %lld, lu_nb %d, ms %.3f\n", kv.first,
                     (long long)kv.second.n_max, kv.second.nb, kv.second.ms);
            out += line;
        }
        snprintf(line, sizeof(line), "workers %d\n", g_workers);
        out += line;
    }
    if (buf && buflen > 0) {
        const int k = std::min<int>((int)out.size(), buflen - 1);
        memcpy(buf, out.data(), k);
        buf[k] = '\0';
    }
    return (int)out.size() + 1;
}

int gir_batch_engine(int nsys, const int64_t* n, const int64_t* lda, const gir_params* params) {
    if (nsys < 1 || !n || !lda || !params) return -1;
    const bool ok = gir::persistent_batch_supported(nsys, n, lda, params);
    if (params->flags & GIR_FLAG_BATCH_PERSISTENT) return ok ? 1 : -1;
    return (ok && gir::persistent_batch_preferred(nsys, n)) ? 1 : 0;
}

gir_status gir_batch_solve(int nsys, const int64_t* n, const double* const* A, const int64_t* lda,
                           const double* const* b, double* const* x, const gir_params* params, gir_info* infos,
                           void* stream) {
    if (nsys < 0 || (nsys > 0 && (!n || !A || !lda || !b || !x || !params))) return GIR_INVALID_ARG;
    if (nsys == 0) return GIR_OK;
    cudaStream_t caller = (cudaStream_t)stream;
    if (params->flags & GIR_FLAG_AUTOTUNE) {
        gir_status t = gir_autotune(n, nsys, caller);
        if (t != GIR_OK) return t;
    }
    const int engine = gir_batch_engine(nsys, n, lda, params);
    if (engine < 0) return GIR_UNSUPPORTED;   // the persistent kernel was asked for and cannot take it
    if (engine == 1) return persistent_batch_solve(nsys, n, A, lda, b, x, params, infos, caller);
    gir_params p = *params;
    p.flags = 0;
    // longest first: the LU is O(n^3), so this keeps the largest systems off the tail
    std::vector<int> order(nsys);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return n[a] > n[c]; });
    int workers;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        workers = g_workers > 0 ? g_workers : 8;
    }
    workers = std::max(1, std::min(workers, nsys));
    int dev = 0;
    cudaGetDevice(&dev);
    cudaEvent_t start;
    cudaEventCreateWithFlags(&start, cudaEventDisableTiming);
    cudaEventRecord(start, caller);
    std::vector<gir_status> status(nsys, GIR_OK);
    std::vector<gir_info> loc(nsys);
    std::atomic<int> next{0};
    std::vector<cudaEvent_t> done(workers);
    std::vector<std::thread> th;
    for (int w = 0; w < workers; ++w) {
        cudaEventCreateWithFlags(&done[w], cudaEventDisableTiming);
        th.emplace_back([&, w]() {
            cudaSetDevice(dev);
            cudaStream_t s;
            cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
            cudaStreamWaitEvent(s, start, 0);
            for (int i = next++; i < nsys; i = next++) {
                const int sys = order[i];
                memset(&loc[sys], 0, sizeof(gir_info));
                gir_handle* h = nullptr;
                gir_status st = gir_factor(A[sys], n[sys], lda[sys], &p, s, &h);
                if (st == GIR_OK) st = gir_solve(h, A[sys], lda[sys], b[sys], x[sys], &loc[sys], s);
                if (h) {
                    cudaStreamSynchronize(s);
                    release_handle_on(h, s);
                }
                loc[sys].status = st;
                status[sys] = st;
            }
            cudaEventRecord(done[w], s);
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        });
    }
    for (auto& t : th) t.join();
    for (int w = 0; w < workers; ++w) {
        cudaStreamWaitEvent(caller, done[w], 0);
        cudaEventDestroy(done[w]);
    }
    cudaEventDestroy(start);
    gir_status worst = GIR_OK;
    for (int i = 0; i < nsys; ++i) {
        if (infos) infos[i] = loc[i];
        const gir_status s = status[i];
        if (s != GIR_OK && (worst == GIR_OK || worst == GIR_NOT_CONVERGED)) worst = s;
    }
    return worst;
}

}  // extern "C"
