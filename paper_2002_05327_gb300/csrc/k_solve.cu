// Subdomain solves of one dependency level of Algorithm 3.1 / 4.1
// ("solve the local solution u^l_ij with the local source r^l_ij").
//
// With the block-Thomas factors D_j = S_j^{-1} of k_factor.cu:
//     forward   y_0 = D_0 b_0,            y_j = D_j (b_j - a_j * y_{j-1})
//     backward  u_{L-1} = y_{L-1},        u_j = y_j - D_j (c_j * u_{j+1})
// with a_j[p] = Pv[p] / alpha_slow(face j), c_j[p] = Pv[p] / alpha_slow(face j+1),
// Pv[p] = prod of the non-slow alphas at block node p over h^2.
//
// Work split: one CTA per (task, panel of PG right-hand sides); thread p owns
// row p of the block for all PG columns.  The right-hand side panel (n x PG)
// sits in shared memory as [q][c].  D_j is stored column-major with split
// planes (column q = nbp reals then nbp imaginaries), so CQ whole columns are
// one contiguous span: thread 0 streams D through a ring of NSTAGE shared
// buffers with cp.async.bulk (the bulk-copy engine) and mbarrier completion,
// running NSTAGE chunks ahead -- across line boundaries and from the forward
// into the backward pass, since D does not depend on the recurrence.  Every
// mbarrier wait is bounded; on expiry the CTA raises the error word, drains
// its copies in flight (bounded) and leaves.
//
// The window buffer holds b on entry, y after the forward pass and u on exit
// (layout [rhs][line][p]).
#include "helm_internal.h"

namespace helm {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// Bounded wait on an mbarrier phase; returns false if the limit expired.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
    uint32_t done = 0;
    for (uint32_t it = 0; it < limit; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

constexpr uint32_t kWaitLimit = 1u << 22;  // try_wait rounds (each suspends up to a time slice)

struct SolveGeom {
    int cq;      // columns per chunk
    int nstage;  // ring depth
};

// Chunk sequence: forward lines 0..L-1 then backward lines L-2..0, each line
// split into ceil(n/cq) chunks of cq columns.
struct ChunkSeq {
    int n, nl, cq, per_line, total;
    __device__ ChunkSeq(int n_, int nl_, int cq_) : n(n_), nl(nl_), cq(cq_) {
        per_line = (n + cq - 1) / cq;
        total = (2 * nl - 1) * per_line;
    }
    __device__ __forceinline__ int line_of(int i) const {
        int li = i / per_line;
        return li < nl ? li : 2 * nl - 2 - li;
    }
    __device__ __forceinline__ int col0(int i) const { return (i % per_line) * cq; }
};

template <typename T, int PG>
__global__ void __launch_bounds__(1024) solve_kernel(const Task* __restrict__ tasks,
                                                     const SubDesc* __restrict__ subs, int nrhs,
                                                     const T* __restrict__ fac,
                                                     const cplx<T>* __restrict__ Pv,
                                                     const cplx<T>* __restrict__ inva,
                                                     cplx<T>* buf, int64_t rstride, SolveGeom G,
                                                     int nbp_max, int* err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const Task tk = tasks[blockIdx.x];
    const SubDesc& S = subs[tk.sub];
    const int n = S.nblk, nbp = S.nbp, nl = S.nlines;
    const int cq = G.cq, NS = G.nstage;
    const size_t stage_elems = (size_t)cq * 2 * nbp_max;
    T* stages = reinterpret_cast<T*>(smem_raw);
    cplx<T>* rs = reinterpret_cast<cplx<T>*>(stages + stage_elems * NS);  // [nbp_max][PG]
    uint64_t* full = reinterpret_cast<uint64_t*>(rs + (size_t)nbp_max * PG);
    __shared__ int abort_flag;

    const int c0 = blockIdx.y * PG;
    const int p = threadIdx.x;
    const bool row = p < n;
    const cplx<T>* pv = Pv + S.coup_off;
    const cplx<T>* ia = inva + S.inva_off;
    const cplx<T> pvp = row ? pv[p] : mk<T>(0, 0);
    cplx<T>* V = buf + tk.buf_off;
    int ncol = nrhs - c0;
    if (ncol > PG) ncol = PG;

    const ChunkSeq seq(n, nl, cq);
    const T* fbase = fac + S.fac_off;
    const size_t line_elems = (size_t)2 * nbp * nbp;
    auto issue = [&](int i) {  // thread 0 only
        const int s = i % NS;
        const int l = seq.line_of(i), q0 = seq.col0(i);
        const int cols = min(cq, n - q0);
        const uint32_t bytes = (uint32_t)(cols * 2 * nbp * sizeof(T));
        mbar_expect_tx(&full[s], bytes);
        bulk_g2s(stages + s * stage_elems, fbase + l * line_elems + (size_t)q0 * 2 * nbp, bytes,
                 &full[s]);
    };
    if (p == 0) {
        abort_flag = 0;
        for (int s = 0; s < NS; ++s) mbar_init(&full[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (p == 0)
        for (int i = 0; i < NS && i < seq.total; ++i) issue(i);

    cplx<T> prev[PG], acc[PG];
#pragma unroll
    for (int c = 0; c < PG; ++c) prev[c] = mk<T>(0, 0);

    int ci = 0;  // next chunk to consume
    bool ok = true;
    // multiply the staged panel rs by D_j, chunk by chunk, into acc
    auto line_gemv = [&]() {
#pragma unroll
        for (int c = 0; c < PG; ++c) acc[c] = mk<T>(0, 0);
        for (int k = 0; k < seq.per_line; ++k, ++ci) {
            const int s = ci % NS;
            const uint32_t parity = (uint32_t)((ci / NS) & 1);
            if (!mbar_wait(&full[s], parity, kWaitLimit)) {
                atomicExch(err, 2);
                abort_flag = 1;
            }
            __syncthreads();
            if (abort_flag) {
                ok = false;
                return;
            }
            const int q0 = seq.col0(ci);
            const int cols = min(cq, n - q0);
            if (row) {
                const T* Dc = stages + s * stage_elems + p;
#pragma unroll 4
                for (int qq = 0; qq < cols; ++qq) {
                    const cplx<T> d = mk<T>(Dc[(size_t)qq * 2 * nbp], Dc[(size_t)qq * 2 * nbp + nbp]);
                    const cplx<T>* r = rs + (size_t)(q0 + qq) * PG;
#pragma unroll
                    for (int c = 0; c < PG; ++c) cfma(acc[c], d, r[c]);
                }
            }
            __syncthreads();
            if (p == 0 && ci + NS < seq.total) issue(ci + NS);
        }
    };

    // ---------------- forward
    for (int j = 0; j < nl && ok; ++j) {
        if (row) {
            cplx<T> a = (j > 0) ? pvp * ia[j] : mk<T>(0, 0);
#pragma unroll
            for (int c = 0; c < PG; ++c) {
                cplx<T> v = mk<T>(0, 0);
                if (c < ncol) v = V[(int64_t)(c0 + c) * rstride + (int64_t)j * n + p] - a * prev[c];
                rs[p * PG + c] = v;
            }
        }
        __syncthreads();
        line_gemv();
        if (!ok) break;
        if (row) {
#pragma unroll
            for (int c = 0; c < PG; ++c) {
                prev[c] = acc[c];
                if (c < ncol) V[(int64_t)(c0 + c) * rstride + (int64_t)j * n + p] = acc[c];
            }
        }
    }
    // ---------------- backward (prev = u_{L-1} = y_{L-1})
    for (int j = nl - 2; j >= 0 && ok; --j) {
        if (row) {
            cplx<T> cc = pvp * ia[j + 1];
#pragma unroll
            for (int c = 0; c < PG; ++c) rs[p * PG + c] = cc * prev[c];
        }
        __syncthreads();
        line_gemv();
        if (!ok) break;
        if (row) {
#pragma unroll
            for (int c = 0; c < PG; ++c) {
                cplx<T> y = (c < ncol) ? V[(int64_t)(c0 + c) * rstride + (int64_t)j * n + p]
                                       : mk<T>(0, 0);
                prev[c] = y - acc[c];
                if (c < ncol) V[(int64_t)(c0 + c) * rstride + (int64_t)j * n + p] = prev[c];
            }
        }
    }
    if (!ok && p == 0) {
        // drain: wait (bounded) for every copy still in flight before leaving
        for (int i = ci; i < seq.total && i < ci + NS; ++i)
            mbar_wait(&full[i % NS], (uint32_t)((i / NS) & 1), kWaitLimit);
    }
}

static SolveGeom geom_for(int nbp_max, size_t esize, int PG, size_t* smem) {
    SolveGeom g;
    const size_t col_bytes = 2 * (size_t)nbp_max * esize;
    g.cq = (int)std::max<size_t>(1, (48 * 1024) / col_bytes);
    const size_t rs_bytes = (size_t)nbp_max * PG * 2 * esize;
    const size_t budget = 200 * 1024;
    g.nstage = 4;
    while (g.nstage > 2 && g.nstage * g.cq * col_bytes + rs_bytes + 64 > budget) --g.nstage;
    while (g.nstage * g.cq * col_bytes + rs_bytes + 64 > budget && g.cq > 1) --g.cq;
    *smem = g.nstage * g.cq * col_bytes + rs_bytes + 8 * g.nstage + 16;
    return g;
}

template <typename T, int PG>
static void launch_pg(const Task* tasks, int ntask, const SubDesc* subs, int nbp_max, int nrhs,
                      const T* fac, const cplx<T>* Pv, const cplx<T>* inva, cplx<T>* buf,
                      int64_t rstride, int* err, cudaStream_t st) {
    size_t smem = 0;
    SolveGeom g = geom_for(nbp_max, sizeof(T), PG, &smem);
    cudaFuncSetAttribute(solve_kernel<T, PG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    dim3 grid(ntask, (nrhs + PG - 1) / PG);
    solve_kernel<T, PG><<<grid, nbp_max, smem, st>>>(tasks, subs, nrhs, fac, Pv, inva, buf,
                                                      rstride, g, nbp_max, err);
}

template <typename T>
void launch_solve(const Task* tasks, int ntask, const SubDesc* subs, int nbp_max, int nrhs,
                  int panel, const T* fac, const cplx<T>* Pv, const cplx<T>* inva, cplx<T>* buf,
                  int64_t rstride, int* err, cudaStream_t st) {
    if (ntask == 0) return;
    switch (panel) {
        case 1: launch_pg<T, 1>(tasks, ntask, subs, nbp_max, nrhs, fac, Pv, inva, buf, rstride, err, st); break;
        case 2: launch_pg<T, 2>(tasks, ntask, subs, nbp_max, nrhs, fac, Pv, inva, buf, rstride, err, st); break;
        case 4: launch_pg<T, 4>(tasks, ntask, subs, nbp_max, nrhs, fac, Pv, inva, buf, rstride, err, st); break;
        default: launch_pg<T, 8>(tasks, ntask, subs, nbp_max, nrhs, fac, Pv, inva, buf, rstride, err, st); break;
    }
}

template void launch_solve<float>(const Task*, int, const SubDesc*, int, int, int, const float*,
                                  const cplx<float>*, const cplx<float>*, cplx<float>*, int64_t,
                                  int*, cudaStream_t);
template void launch_solve<double>(const Task*, int, const SubDesc*, int, int, int,
                                   const double*, const cplx<double>*, const cplx<double>*,
                                   cplx<double>*, int64_t, int*, cudaStream_t);

}  // namespace helm
