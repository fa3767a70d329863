// Application of the LU preconditioner M^-1 = mu S U^-1 L^-1 P R (Algorithm 4, correction equation) and of
// its transpose, on the u_f factors, with float-float arithmetic (about 48 significand bits).
//
// Triangular solves are blocked by b = 64 rows. One persistent CTA per block row takes a
// ticket (atomic counter) in solve order; it streams the off-diagonal tiles of its block row
// as the solution elements it depends on are published, then multiplies by the precomputed
// inverse of its diagonal block and publishes its own block. A CTA only waits for tickets
// smaller than its own, which belong to CTAs that are already running, so the scheme cannot
// deadlock; every wait is bounded and a timeout sets an abort flag that releases all waiters.
#include "gir_internal.cuh"
#include "k_trsv.cuh"
#include "trace.cuh"

namespace gir {

constexpr int TB = TRSV_BLOCK;  // 64

// ------------------------------------------------------------------ diagonal-block inverses
// D[I] = inv(T_II) for T = L (unit lower, upper == 0) or U (upper == 1), computed in FP64 from
// the u_f values and stored as float-float (row-major b x b per block). Rows/columns beyond n
// are padded with the identity.
__global__ void __launch_bounds__(TB) k_diag_inv(const uint16_t* __restrict__ LU, int64_t ldl, int64_t n, int fmt,
                                                 int upper, float2* __restrict__ D) {
    extern __shared__ double dsm[];
    double (*T)[TB + 1] = reinterpret_cast<double (*)[TB + 1]>(dsm);
    double (*X)[TB + 1] = reinterpret_cast<double (*)[TB + 1]>(dsm + TB * (TB + 1));
    const int I = blockIdx.x;
    const int64_t base = (int64_t)I * TB;
    const int c = threadIdx.x;
    for (int i = 0; i < TB; ++i) {
        int64_t gi = base + i, gc = base + c;
        double v;
        if (gi < n && gc < n) {
            v = (double)uf_to_float(LU[gi * ldl + gc], fmt);
            if (!upper) v = (c < i) ? v : (c == i ? 1.0 : 0.0);
            else v = (c >= i) ? v : 0.0;
        } else {
            v = (i == c) ? 1.0 : 0.0;
        }
        T[i][c] = v;
    }
    __syncthreads();
    // thread c solves T x = e_c
    if (!upper) {
        for (int i = 0; i < TB; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int q = 0; q < i; ++q) s = fma(-T[i][q], X[q][c], s);
            X[i][c] = s;
        }
    } else {
        for (int i = TB - 1; i >= 0; --i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int q = i + 1; q < TB; ++q) s = fma(-T[i][q], X[q][c], s);
            X[i][c] = s / T[i][i];
        }
    }
    __syncthreads();
    for (int i = 0; i < TB; ++i) {
        double v = X[i][c];
        float h = __double2float_rn(v);
        float l = __double2float_rn(v - (double)h);
        D[((int64_t)I * TB + i) * TB + c] = make_float2(h, l);
    }
}

// E[I] = D'[I] T'_{I,J}: the product of the diagonal-block inverse with the block that a solve meets
// last, J = I + 1 (next == 1: backward order) or I - 1 (next == 0: forward order). For M^-1
// (trans == 0) D' and T' are the stored blocks (L solve: DL, J = I - 1; U solve: DU, J = I + 1); for
// M^-T (trans == 1) they are the transposes (U^T solve: DU^T with T'_{I,J} = U_{J,I}^T, J = I - 1;
// L^T solve: DL^T with T'_{I,J} = L_{J,I}^T, J = I + 1). Float-float dot products of the float-float
// D with the u_f tile (exact in FP32), stored as float-float (row-major b x b per block, in the
// solve's own orientation); blocks without such a neighbour, and rows/columns beyond n, are zero.
__global__ void __launch_bounds__(256) k_diag_e(const uint16_t* __restrict__ LU, int64_t ldl, int64_t n, int fmt,
                                                int next, int trans, const float2* __restrict__ D, int nblk,
                                                float2* __restrict__ E) {
    __shared__ float2 Ds[TB][TB + 1];
    __shared__ uint16_t Ts[TB][TB + 2];
    const int I = blockIdx.x;
    const int J = next ? I + 1 : I - 1;
    const int tid = threadIdx.x;
    float2* Eb = E + (int64_t)I * TB * TB;
    if (J < 0 || J >= nblk) {
        for (int e = tid; e < TB * TB; e += 256) Eb[e] = make_float2(0.0f, 0.0f);
        return;
    }
    for (int e = tid; e < TB * TB; e += 256) {
        const int i = e / TB, c = e % TB;
        if (!trans) {
            Ds[i][c] = D[(int64_t)I * TB * TB + e];
            const int64_t gi = (int64_t)I * TB + i, gc = (int64_t)J * TB + c;
            Ts[i][c] = (gi < n && gc < n) ? LU[gi * ldl + gc] : (uint16_t)0;   // 0 is +0 in both formats
        } else {
            Ds[c][i] = D[(int64_t)I * TB * TB + e];
            const int64_t gr = (int64_t)J * TB + c, gc = (int64_t)I * TB + i;
            Ts[i][c] = (gr < n && gc < n) ? LU[gr * ldl + gc] : (uint16_t)0;
        }
    }
    __syncthreads();
    const int r = tid >> 2, q = tid & 3;
    for (int c = q * 16; c < q * 16 + 16; ++c) {
        float sh = 0.0f, sl = 0.0f;
        for (int k = 0; k < TB; ++k) {
            const float2 d = Ds[r][k];
            ff_acc_prod1(sh, sl, uf_to_float(Ts[k][c], fmt), d.x, d.y);
        }
        const ff v = ff_norm(sh, sl);
        const bool live = (int64_t)I * TB + r < n && (int64_t)J * TB + c < n;
        Eb[r * TB + c] = live ? make_float2(v.h, v.l) : make_float2(0.0f, 0.0f);
    }
}

// ------------------------------------------------------------------ persistent block TRSV
__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// Output y (float-float) is published element by element: y starts as the all-ones pattern (an
// FP32 NaN no computation writes) and each element is written with one 64-bit store, so a
// consumer polls the data itself instead of a separate flag.
constexpr unsigned long long Y_EMPTY = 0xFFFFFFFFFFFFFFFFull;

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long pack_ff(float h, float l) {
    if (h != h) h = __int_as_float(0x7fc00000);  // canonical NaN, never the empty pattern
    if (l != l) l = 0.0f;
    return ((unsigned long long)__float_as_uint(l) << 32) | (unsigned long long)__float_as_uint(h);
}

// ------------------------------------------------------------------ pre/post scaling
// forward: z[i] = R[p] * w[p], p = perm[i]          (P R w)
__global__ void k_minv_pre(const double* __restrict__ w, const int* __restrict__ perm, const double* __restrict__ R,
                           int64_t n, double* __restrict__ z) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t p = perm[i];
        z[i] = R ? R[p] * w[p] : w[p];
    }
}
// transpose: z = S w
__global__ void k_minv_pre_t(const double* __restrict__ w, const double* __restrict__ S, int64_t n,
                             double* __restrict__ z) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        z[i] = S ? S[i] * w[i] : w[i];
}
// forward: out[i] = fl_u(mu S[i] y[i])
__global__ void k_minv_post(const float2* __restrict__ y, const double* __restrict__ S, double mu, int64_t n,
                            int round32, double* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = (double)y[i].x + (double)y[i].y;
        if (S) v *= S[i] * mu;
        if (round32) v = (double)__double2float_rn(v);
        out[i] = v;
    }
}
// transpose: out[perm[i]] = fl_u(mu R[perm[i]] y[i])
__global__ void k_minv_post_t(const float2* __restrict__ y, const int* __restrict__ perm, const double* __restrict__ R,
                              double mu, int64_t n, int round32, double* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t p = perm[i];
        double v = (double)y[i].x + (double)y[i].y;
        if (R) v *= R[p] * mu;
        if (round32) v = (double)__double2float_rn(v);
        out[p] = v;
    }
}

// ------------------------------------------------------------------ forward-order solves
// M^-1 applies L then U in their natural orders (TRANS = false). Same 64-row blocks as k_trsv,
// organised for latency: 256 threads, row r = tid / 4 of the block and quarter q = tid % 4 of
// its columns (16 each). The off-diagonal tiles do not depend on y, so they stream through a
// 4-stage cp.async ring (each thread copies and later reads only its own 32 bytes of a tile) and
// a CTA that falls behind the published blocks catches up at streaming speed; the four lanes of
// a row reduce by shuffles and all hold the row's accumulator, so each tile costs one CTA
// barrier (for the shared block of y).
//
// Consecutive blocks form a thread-block cluster (TF_CLUSTER CTAs, one ticket per cluster). A
// finished block is published to global memory for later clusters and, in parallel, pushed into
// the shared memory of the later CTAs of its own cluster with st.async, counted on one mbarrier
// per source block: a dependency inside the cluster arrives in about 0.12 us, against about
// 0.86 us for a release/acquire hop through global memory, and the chain of blocks crosses
// global memory only once per cluster.
constexpr int TF_STAGES = 4;
constexpr int TF_AHEAD = TF_STAGES - 1;
constexpr size_t TF_DYN_SMEM = (size_t)TF_STAGES * (2 * 256 * 16 + 64 * 8);
constexpr int TF_MAXCL = 16;
constexpr long long TF_WAIT_LIMIT = 20000000LL;   // polls of one in-cluster dependency

__device__ __forceinline__ void tf_cp_async16(void* smem, const void* gmem, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void tf_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void tf_cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ uint32_t tf_cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t tf_cluster_size() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void tf_cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t tf_map(const void* p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(r)
                 : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ void tf_mbar_init(unsigned long long* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(bar)) : "memory");
}
__device__ __forceinline__ void tf_mbar_expect(unsigned long long* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool tf_mbar_test(unsigned long long* bar) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], 0;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"((uint32_t)__cvta_generic_to_shared(bar))
        : "memory");
    return done != 0;
}
__device__ __forceinline__ void tf_st_async_u64(uint32_t addr, unsigned long long v, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.b32 [%0], {%1, %2}, [%3];" ::"r"(addr),
                 "r"((uint32_t)(v & 0xffffffffull)), "r"((uint32_t)(v >> 32)), "r"(bar)
                 : "memory");
}

// TRANS: the solve of M^-T meets block (I, J) as the transpose of stored block (J, I). A thread then
// copies 32 bytes of row r of the stored tile (J, I) (contiguous, like the forward case), which
// contribute to 16 different solution rows: it keeps 16 float-float partial sums across all the
// dependencies, and the 64 rows of the tile are summed once per block (shuffles within a warp, one
// shared-memory pass across warps) while the block still waits for its last dependency. D and E
// arrive in the solve's own orientation for E and stored orientation for D (read transposed).
template <bool LOWER, bool TRANS>
__device__ __forceinline__ void trsv_cluster_body(const uint16_t* __restrict__ LU, int64_t ldl, int fmt,
                                                  const float2* __restrict__ D, const float2* __restrict__ E,
                                                  int64_t n, int nblk,
                                                  const double* __restrict__ zin64, const float2* __restrict__ zin_ff,
                                                  float2* __restrict__ yout, unsigned long long* __restrict__ ticket_ctr,
                                                  unsigned long long base, int* __restrict__ abort_flag,
                                                  int* __restrict__ flags) {
    // dynamic: the ring of tiles [stage][chunk][thread] and the y blocks fetched ahead [stage][TB]
    extern __shared__ __align__(16) unsigned char tf_dyn[];
    uint4 (*ring)[2][256] = reinterpret_cast<uint4 (*)[2][256]>(tf_dyn);
    unsigned long long (*ring_y)[TB] =
        reinterpret_cast<unsigned long long (*)[TB]>(tf_dyn + (size_t)TF_STAGES * 2 * 256 * sizeof(uint4));
    __shared__ float2 yj[2][TB + 2];                          // padded by one entry per 32
    __shared__ float2 accs[TB + 2];
    __shared__ float2 wred[TRANS ? 8 : 1][TB + 2];              // TRANS: per-warp sums of the tile rows
    __shared__ __align__(8) unsigned long long cbar[TF_MAXCL];               // one per lower rank
    __shared__ __align__(16) unsigned long long ycl[TF_MAXCL][TB];           // blocks of lower ranks
    __shared__ int s_ticket, s_abort;
    unsigned long long* ybits = reinterpret_cast<unsigned long long*>(yout);
    const int tid = threadIdx.x;
    const int crank = (int)tf_cluster_rank(), csize = (int)tf_cluster_size();
    if (tid == 0) {
        s_abort = 0;
        for (int i = 0; i < crank; ++i) tf_mbar_init(&cbar[i]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int i = 0; i < crank; ++i) tf_mbar_expect(&cbar[i], TB * 8);
    }
    tf_cluster_sync();   // every CTA of the cluster runs, with its barriers armed
    if (crank == 0 && tid == 0) {
        const int kc = (int)(atomicAdd(ticket_ctr, 1ULL) - base);
        for (int r = 0; r < csize; ++r)
            asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(tf_map(&s_ticket, (uint32_t)r)), "r"(kc) : "memory");
    }
    tf_cluster_sync();   // the cluster's ticket is visible
    const int kc = s_ticket;
    const int nclu = (nblk + csize - 1) / csize;
    const int t = kc * csize + crank;           // position of this block in the solve order
    const bool bad = (kc < 0 || kc >= nclu);
    if (bad && tid == 0) { atomicOr(flags, DEV_TIMEOUT); atomicExch(abort_flag, 1); }
    if (!bad && t < nblk) {
        const int I = LOWER ? t : (nblk - 1 - t);
        const int64_t r0 = (int64_t)I * TB;
        const int r = tid >> 2, q = tid & 3;
        const int64_t gi = r0 + r;
        auto pad = [](int c) { return c + (c >> 5); };
        float ah = 0.0f, al = 0.0f;
        if (gi < n) {
            if (zin64) {
                const double v = zin64[gi];
                ah = __double2float_rn(v);
                al = __double2float_rn(v - (double)ah);
            } else {
                const float2 v = zin_ff[gi];
                ah = v.x;
                al = v.y;
            }
        }
        const int ndep = t;                      // every earlier block in the solve order
        const int first_local = kc * csize;      // dependencies from here on come from this cluster
        // this thread's 16 entries of the diagonal-block inverse, loaded now: the product with them
        // follows the last dependency and is on the critical path of the solve
        // (TRANS: loaded after the dependency loop, which holds 16 partial sums in registers)
        float4 dreg[8];
        auto load_d = [&]() {
            if (!TRANS) {
                const float4* drow = reinterpret_cast<const float4*>(D + ((int64_t)I * TB + r) * TB + q * 16);
#pragma unroll
                for (int k = 0; k < 8; ++k) dreg[k] = drow[k];
            } else {
                // entries (q*16 + c, r) of the stored inverse: row r of its transpose
                const float2* dcol = D + ((int64_t)I * TB + q * 16) * TB + r;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float2 d0 = dcol[(2 * k) * TB], d1 = dcol[(2 * k + 1) * TB];
                    dreg[k] = make_float4(d0.x, d0.y, d1.x, d1.y);
                }
            }
        };
        if (!TRANS) load_d();
        // and its 16 entries of E = D_I T_{I,J} for the last dependency J: once y_J arrives, only
        // y_I = w - E y_J remains, with w = D_I (z_I - sum over the other dependencies) formed
        // while the block still waits
        float4 ereg[8];
        {
            const float4* erow = reinterpret_cast<const float4*>(E + ((int64_t)I * TB + r) * TB + q * 16);
#pragma unroll
            for (int k = 0; k < 8; ++k) ereg[k] = ndep > 0 ? erow[k] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        auto dep_block = [&](int step) { return LOWER ? step : (nblk - 1 - step); };
        // the tile of a dependency and, for a block of an earlier cluster, its y values (read at
        // L2 by cp.async.cg): a block published before its step comes up costs no round trip
        auto issue = [&](int step, int st) {
            const int J = dep_block(step);
            // forward: row gi of the stored tile (I, J); TRANS: row r of the stored tile (J, I)
            const int64_t trow = TRANS ? (int64_t)J * TB + r : gi;
            const int64_t c0 = (TRANS ? r0 : (int64_t)J * TB) + q * 16;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int64_t cc = c0 + 8 * k;
                int bytes = 0;
                if (trow < n && cc < n && step < ndep - 1) bytes = (int)(2 * gmin<int64_t>(8, n - cc));
                const uint16_t* src = bytes ? LU + trow * ldl + cc : LU;
                tf_cp_async16(&ring[st][k][tid], src, bytes);
            }
            if (step < first_local && tid < TB / 2) {
                const int64_t e = (int64_t)J * TB + 2 * tid;   // two 8-byte values per thread
                const int bytes = (int)(8 * gmin<int64_t>(2, gmax<int64_t>(0, n - e)));
                tf_cp_async16(&ring_y[st][2 * tid], bytes ? (const void*)(ybits + e) : (const void*)ybits, bytes);
            }
        };
        // each of threads 0..31 reads the two values its own cp.async fetched (no other thread's
        // copy is read before a barrier), polling global memory only for a value still unpublished
        auto wait_global = [&](int J, int buf, int st) {
            if (tid < TB / 2) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int e = 2 * tid + h;
                    const int64_t gc = (int64_t)J * TB + e;
                    unsigned long long v = ring_y[st][e];
                    if (gc < n && v == Y_EMPTY) {
                        long long spins = 0;
                        while ((v = ld_relaxed_u64(ybits + gc)) == Y_EMPTY) {
                            if (((spins & 1023) == 0) && ld_acquire(abort_flag)) { s_abort = 1; break; }
                            if (++spins > SPIN_LIMIT) {
                                atomicOr(flags, DEV_TIMEOUT);
                                atomicExch(abort_flag, 1);
                                s_abort = 1;
                                break;
                            }
                        }
                    }
                    if (gc >= n) v = 0ull;
                    yj[buf][pad(e)] = make_float2(__uint_as_float((unsigned)(v & 0xffffffffull)),
                                                  __uint_as_float((unsigned)(v >> 32)));
                }
            }
        };
        auto wait_local = [&](int src, int buf) {
            if (tid < TB) {
                long long spins = 0;
                bool ok = true;
                while (!tf_mbar_test(&cbar[src])) {
                    if (((spins & 1023) == 0) && ld_acquire(abort_flag)) { ok = false; break; }
                    if (++spins > TF_WAIT_LIMIT) {
                        atomicOr(flags, DEV_TIMEOUT);
                        atomicExch(abort_flag, 1);
                        ok = false;
                        break;
                    }
                }
                const unsigned long long v = ok ? ycl[src][tid] : 0ull;
                if (!ok) s_abort = 1;
                yj[buf][pad(tid)] = make_float2(__uint_as_float((unsigned)(v & 0xffffffffull)),
                                                __uint_as_float((unsigned)(v >> 32)));
            }
        };
        auto quad_reduce = [&](float& sh, float& sl) {
#pragma unroll
            for (int o = 1; o <= 2; o <<= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, sh, o);
                const float ol = __shfl_xor_sync(0xffffffffu, sl, o);
                ff_acc_add(sh, sl, oh, ol);
            }
        };
        float part_h[TRANS ? 16 : 1], part_l[TRANS ? 16 : 1];   // TRANS: sums for rows q*16 + c
#pragma unroll
        for (int c = 0; c < (TRANS ? 16 : 1); ++c) part_h[c] = part_l[c] = 0.0f;
#pragma unroll
        for (int p = 0; p < TF_AHEAD; ++p) {
            if (p < ndep) issue(p, p);
            tf_cp_commit();
        }
        for (int step = 0; step < ndep - 1; ++step) {
            if (step + TF_AHEAD < ndep) issue(step + TF_AHEAD, (step + TF_AHEAD) % TF_STAGES);
            tf_cp_commit();
            tf_cp_wait<TF_AHEAD>();
            const int buf = step & 1;
            const int st = step % TF_STAGES;
            if (step >= first_local) wait_local(step - first_local, buf);
            else wait_global(dep_block(step), buf, st);
            __syncthreads();
            if (s_abort) break;
            if (TRANS) {
                const float2 yv = yj[buf][pad(r)];
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const uint4 v = ring[st][k][tid];
                    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const int c = 8 * k + 2 * m;
                        ff_acc_prod1(part_h[c], part_l[c], uf_to_float((uint16_t)(w[m] & 0xffffu), fmt), yv.x, yv.y);
                        ff_acc_prod1(part_h[c + 1], part_l[c + 1], uf_to_float((uint16_t)(w[m] >> 16), fmt), yv.x,
                                     yv.y);
                    }
                }
                if ((step & 3) == 3) {
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        const ff ns = ff_norm(part_h[c], part_l[c]);
                        part_h[c] = ns.h;
                        part_l[c] = ns.l;
                    }
                }
                continue;
            }
            // two partial sums: half-length dependency chains
            float sh = 0.0f, sl = 0.0f, th = 0.0f, tl = 0.0f;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const uint4 v = ring[st][k][tid];
                const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const int c = q * 16 + 8 * k + 2 * m;
                    const float2 y0 = yj[buf][pad(c)], y1 = yj[buf][pad(c + 1)];
                    ff_acc_prod1(sh, sl, uf_to_float((uint16_t)(w[m] & 0xffffu), fmt), y0.x, y0.y);
                    ff_acc_prod1(th, tl, uf_to_float((uint16_t)(w[m] >> 16), fmt), y1.x, y1.y);
                }
            }
            ff_acc_add(sh, sl, th, tl);
            quad_reduce(sh, sl);
            ff_acc_add(ah, al, -sh, -sl);
            const ff ns = ff_norm(ah, al);
            ah = ns.h;
            al = ns.l;
        }
        if (TRANS) {
            load_d();
            // sum the partial sums over the 64 tile rows: the 8 rows of a warp by shuffles, then the
            // 8 warps through shared memory into the accumulator of row r (threads with q == 0)
#pragma unroll
            for (int o = 4; o <= 16; o <<= 1) {
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const float oh = __shfl_xor_sync(0xffffffffu, part_h[c], o);
                    const float ol = __shfl_xor_sync(0xffffffffu, part_l[c], o);
                    ff_acc_add(part_h[c], part_l[c], oh, ol);
                }
            }
            if ((tid & 31) < 4) {
#pragma unroll
                for (int c = 0; c < 16; ++c) wred[tid >> 5][pad(q * 16 + c)] = make_float2(part_h[c], part_l[c]);
            }
            __syncthreads();
            if (q == 0) {
#pragma unroll
                for (int wp = 0; wp < 8; ++wp) {
                    const float2 v = wred[wp][pad(r)];
                    ff_acc_add(ah, al, -v.x, -v.y);
                }
                const ff ns = ff_norm(ah, al);
                ah = ns.h;
                al = ns.l;
            }
        }
        // w = D_I acc (acc holds everything but the last dependency)
        if (q == 0) accs[pad(r)] = make_float2(ah, al);
        __syncthreads();
        float ph = 0.0f, pl = 0.0f, qh = 0.0f, ql = 0.0f;
        {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float4 d = dreg[k];   // two float-float entries
                const float2 a0 = accs[pad(q * 16 + 2 * k)], a1 = accs[pad(q * 16 + 2 * k + 1)];
                ff_acc_prod2(ph, pl, d.x, d.y, a0.x, a0.y);
                ff_acc_prod2(qh, ql, d.z, d.w, a1.x, a1.y);
            }
            ff_acc_add(ph, pl, qh, ql);
            quad_reduce(ph, pl);
        }
        if (ndep > 0 && !s_abort) {
            // the last dependency: y_I = w - E y_J
            const int step = ndep - 1;
            tf_cp_wait<0>();
            const int buf = step & 1;
            const int st = step % TF_STAGES;
            if (step >= first_local) wait_local(step - first_local, buf);
            else wait_global(dep_block(step), buf, st);
            __syncthreads();
            float sh = 0.0f, sl = 0.0f, th = 0.0f, tl = 0.0f;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float4 e = ereg[k];
                const float2 y0 = yj[buf][pad(q * 16 + 2 * k)], y1 = yj[buf][pad(q * 16 + 2 * k + 1)];
                ff_acc_prod2(sh, sl, e.x, e.y, y0.x, y0.y);
                ff_acc_prod2(th, tl, e.z, e.w, y1.x, y1.y);
            }
            ff_acc_add(sh, sl, th, tl);
            quad_reduce(sh, sl);
            ff_acc_add(ph, pl, -sh, -sl);
        }
        tf_cp_wait<0>();
        if (q == 0) {
            const ff ns = ff_norm(ph, pl);
            const unsigned long long packed = s_abort ? pack_ff(0.0f, 0.0f) : pack_ff(ns.h, ns.l);
            // later blocks of this cluster first (their wait is the shortest), then global memory
            for (int dst = crank + 1; dst < csize; ++dst) {
                if (kc * csize + dst >= nblk) break;
                tf_st_async_u64(tf_map(&ycl[crank][r], (uint32_t)dst), packed, tf_map(&cbar[crank], (uint32_t)dst));
            }
            if (gi < n) st_relaxed_u64(ybits + gi, packed);
        }
        // after an abort some messages of lower ranks may still be on their way: take them in
        // (bounded) so that no st.async targets this CTA after it has left
        if (s_abort && tid == 0) {
            for (int i = 0; i < crank; ++i)
                for (long long it = 0; it < TF_WAIT_LIMIT && !tf_mbar_test(&cbar[i]); ++it) {
                }
        }
    }
    // no CTA leaves while a later CTA of its cluster may still be sending to it
    tf_cluster_sync();
}

#define TRSV_CLUSTER_ARGS                                                                                         \
    const uint16_t *__restrict__ LU, int64_t ldl, int fmt, const float2 *__restrict__ D,                        \
        const float2 *__restrict__ E, int64_t n, int nblk, const double *__restrict__ zin64,                    \
        const float2 *__restrict__ zin_ff, float2 *__restrict__ yout, unsigned long long *__restrict__ ticket_ctr, \
        unsigned long long base, int *__restrict__ abort_flag, int *__restrict__ flags
// M^-1's solves: L (LOWER) then U
template <bool LOWER>
__global__ void __launch_bounds__(256) k_trsv_fwd(TRSV_CLUSTER_ARGS) {
    trsv_cluster_body<LOWER, false>(LU, ldl, fmt, D, E, n, nblk, zin64, zin_ff, yout, ticket_ctr, base, abort_flag,
                                    flags);
}
// M^-T's solves: U^T (LOWER: forward order) then L^T (backward order)
template <bool LOWER>
__global__ void __launch_bounds__(256) k_trsv_adj(TRSV_CLUSTER_ARGS) {
    trsv_cluster_body<LOWER, true>(LU, ldl, fmt, D, E, n, nblk, zin64, zin_ff, yout, ticket_ctr, base, abort_flag,
                                   flags);
}
#undef TRSV_CLUSTER_ARGS

// ------------------------------------------------------------------ host side
gir_status trsv_setup(TrsvState& st, const uint16_t* LU, int64_t ldl, int64_t n, int fmt, cudaStream_t s) {
    st.n = n;
    st.nblk = (int)((n + TB - 1) / TB);
    st.fmt = fmt;
    st.LU = LU;
    st.ldl = ldl;
    const int smem = 2 * TB * (TB + 1) * (int)sizeof(double);
    GIR_CUDA_TRY(cudaFuncSetAttribute(k_diag_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const void* kernels[4] = {(const void*)k_trsv_fwd<true>, (const void*)k_trsv_fwd<false>,
                              (const void*)k_trsv_adj<true>, (const void*)k_trsv_adj<false>};
    for (const void* fn : kernels)
        GIR_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TF_DYN_SMEM));
    if (st.cluster > 8) {
        // 16-CTA clusters are a non-portable size: use them only where the device can hold one
        int ok = 1;
        for (int kf = 0; kf < 4 && ok; ++kf) {
            const void* fn = kernels[kf];
            if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
                ok = 0;
                break;
            }
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)st.cluster, 1, 1);
            cfg.blockDim = dim3(256, 1, 1);
            cfg.dynamicSmemBytes = TF_DYN_SMEM;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = (unsigned)st.cluster;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int nclusters = 0;
            if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess || nclusters < 1) ok = 0;
        }
        if (!ok) {
            cudaGetLastError();
            st.cluster = 8;
        }
    }
    count_launch(), k_diag_inv<<<st.nblk, TB, smem, s>>>(LU, ldl, n, fmt, 0, st.DL);
    count_launch(), k_diag_inv<<<st.nblk, TB, smem, s>>>(LU, ldl, n, fmt, 1, st.DU);
    count_launch(), k_diag_e<<<st.nblk, 256, 0, s>>>(LU, ldl, n, fmt, 0, 0, st.DL, st.nblk, st.EL);
    count_launch(), k_diag_e<<<st.nblk, 256, 0, s>>>(LU, ldl, n, fmt, 1, 0, st.DU, st.nblk, st.EU);
    st.et_ready = false;   // the transposed solves' E blocks follow on their first use
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

template <bool LOWER, bool TRANS>
static gir_status run_trsv_cl(TrsvState& st, const float2* D, const float2* E, const double* z64, const float2* zff,
                               float2* y, int* flags, cudaStream_t s) {
    const int csize = st.cluster;
    const int nclu = (st.nblk + csize - 1) / csize;
    unsigned long long base = st.tickets;
    st.tickets += (unsigned long long)nclu;   // one ticket per cluster
    GIR_CUDA_TRY(cudaMemsetAsync(y, 0xFF, (size_t)st.n * sizeof(float2), s));
    const char* name = TRANS ? "trsv adjoint" : "trsv";
    const int tslot = trace_begin(s, name);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nclu * csize), 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = TF_DYN_SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launch();
    GIR_CUDA_TRY(cudaLaunchKernelEx(&cfg, TRANS ? k_trsv_adj<LOWER> : k_trsv_fwd<LOWER>, st.LU, st.ldl, st.fmt, D, E, st.n, st.nblk, z64, zff, y,
                                    st.ticket_ctr, base, st.abort_flag, flags));
    trace_end(tslot, name, s);
    st.calls++;
    return GIR_OK;
}

gir_status apply_minv(TrsvState& st, const double* w, double* out, const double* R, const double* S, double mu,
                      int trans, int round32, int* flags, cudaStream_t s) {
    const int64_t n = st.n;
    const int g = (int)gmin<int64_t>((n + 255) / 256, 1024);
    if (!trans) {
        count_launch(), k_minv_pre<<<g, 256, 0, s>>>(w, st.perm, R, n, st.z);
        GIR_TRY((run_trsv_cl<true, false>(st, st.DL, st.EL, st.z, nullptr, st.y1, flags, s)));
        GIR_TRY((run_trsv_cl<false, false>(st, st.DU, st.EU, nullptr, st.y1, st.y2, flags, s)));
        count_launch(), k_minv_post<<<g, 256, 0, s>>>(st.y2, S, mu, n, round32, out);
    } else {
        if (!st.et_ready) {
            // E'[I] = DU[I]^T U[I-1, I]^T (U^T solve) and DL[I]^T L[I+1, I]^T (L^T solve)
            count_launch(), k_diag_e<<<st.nblk, 256, 0, s>>>(st.LU, st.ldl, n, st.fmt, 0, 1, st.DU, st.nblk, st.EUt);
            count_launch(), k_diag_e<<<st.nblk, 256, 0, s>>>(st.LU, st.ldl, n, st.fmt, 1, 1, st.DL, st.nblk, st.ELt);
            st.et_ready = true;
        }
        count_launch(), k_minv_pre_t<<<g, 256, 0, s>>>(w, S, n, st.z);
        // M^-T = mu R P^T L^-T U^-T S: first U^T (lower), then L^T (upper, unit)
        GIR_TRY((run_trsv_cl<true, true>(st, st.DU, st.EUt, st.z, nullptr, st.y1, flags, s)));
        GIR_TRY((run_trsv_cl<false, true>(st, st.DL, st.ELt, nullptr, st.y1, st.y2, flags, s)));
        count_launch(), k_minv_post_t<<<g, 256, 0, s>>>(st.y2, st.perm, R, mu, n, round32, out);
    }
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

}  // namespace gir
