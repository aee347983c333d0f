// Subdomain solves of one dependency level of Algorithm 3.1 / 4.1
// ("solve the local solution u^l_ij with the local source r^l_ij").
//
// With the block-Thomas factors D_j = S_j^{-1} of k_factor.cu:
//     forward   y_0 = D_0 b_0,            y_j = D_j (b_j - a_j * y_{j-1})
//     backward  u_{L-1} = y_{L-1},        u_j = y_j - D_j (c_j * u_{j+1})
// with a_j[p] = Pv[p] / alpha_slow(face j), c_j[p] = Pv[p] / alpha_slow(face j+1),
// Pv[p] = prod of the non-slow alphas at block node p over h^2.
//
// One CTA per (task, panel of PG right-hand sides).  Consumer threads own
// RPT rows of the block each, for all PG columns; one producer warp streams D.
// D_j is stored column-major with split planes (column q = nbp reals then nbp
// imaginaries), so cq whole columns form one contiguous span: the producer
// copies them with cp.async.bulk into a ring of NS shared stages (full
// barrier: bytes landed; empty barrier: every consumer warp is done with the
// stage), running ahead across line boundaries and from the forward into the
// backward pass (D does not depend on the recurrence).  The right-hand side
// panel of line j (n x PG, [q][c]) is double-buffered, so each line needs a
// single barrier among the consumers.  The global operands of the next step
// (b_{j+1} forward, y_j backward) are loaded before the block product so
// their latency hides behind it.
//
// Every mbarrier wait is bounded.  On expiry the CTA raises the device error
// word, stops issuing copies, finishes the line without further waits,
// drains the copies still in flight (bounded) and leaves.
//
// The window buffer holds b on entry, y after the forward pass and u on exit
// (layout [rhs][line][p]).
#include <algorithm>

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
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// Bounded wait for the completion of the phase with the given parity.
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
// Barrier among the consumer threads that also ORs a flag across them, so
// every consumer takes the same abort decision.
__device__ __forceinline__ bool consumers_sync_any(int nthreads, int flag) {
    uint32_t out;
    asm volatile(
        "{\n\t.reg .pred q, p;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, 1, %2, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(out)
        : "r"(flag), "r"(nthreads)
        : "memory");
    return out != 0;
}

constexpr uint32_t kWaitLimit = kDrainPolls;

struct SolveGeom {
    int cq;       // columns per chunk
    int nstage;   // ring depth
    int ncons;    // consumer threads (multiple of 32)
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

template <typename T, int PG, int RPT>
__global__ void __launch_bounds__(1024) solve_kernel(const Task* __restrict__ tasks,
                                                     const SubDesc* __restrict__ subs, int nrhs,
                                                     const T* __restrict__ fac,
                                                     const cplx<T>* __restrict__ Pv,
                                                     const cplx<T>* __restrict__ inva,
                                                     cplx<T>* buf, const cplx<T>* __restrict__ bsrc,
                                                     int64_t rstride, SolveGeom G, int nbp_max,
                                                     DevStatus ds) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const Task tk = tasks[blockIdx.x];
    const SubDesc& S = subs[tk.sub];
    const int n = S.nblk, nbp = S.nbp, nl = S.nlines;
    const int cq = G.cq, NS = G.nstage, NC = G.ncons;
    const size_t stage_elems = (size_t)cq * 2 * nbp_max;
    T* stages = reinterpret_cast<T*>(smem_raw);
    cplx<T>* rs = reinterpret_cast<cplx<T>*>(stages + stage_elems * NS);  // [2][nbp_max][PG]
    uint64_t* full = reinterpret_cast<uint64_t*>(rs + (size_t)2 * nbp_max * PG);
    uint64_t* empty = full + NS;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + NS);

    const ChunkSeq seq(n, nl, cq);
    const int tid = threadIdx.x;
    const int ncw = NC / 32;
    if (tid == 0) {
        *abort_flag = 0;
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], ncw);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // ======================================================= producer warp
    if (tid >= NC) {
        if (tid != NC) return;
        const T* fbase = fac + S.fac_off;
        const size_t line_elems = (size_t)2 * nbp * nbp;
        int issued = 0;
        for (int i = 0; i < seq.total; ++i) {
            const int s = i % NS;
            if (i >= NS && !mbar_wait(&empty[s], (uint32_t)(((i / NS) - 1) & 1), ds.polls)) {
                atomicExch(ds.err, 2);
                *abort_flag = 1;
            }
            if (*abort_flag) break;
            const int l = seq.line_of(i), q0 = seq.col0(i);
            const int cols = min(cq, n - q0);
            const uint32_t bytes = (uint32_t)(cols * 2 * nbp * sizeof(T));
            mbar_expect_tx(&full[s], bytes);
            bulk_g2s(stages + s * stage_elems, fbase + l * line_elems + (size_t)q0 * 2 * nbp, bytes,
                     &full[s]);
            issued = i + 1;
        }
        // drain: every issued copy must land before the CTA's shared memory is released
        for (int i = max(0, issued - NS); i < issued; ++i)
            mbar_wait(&full[i % NS], (uint32_t)((i / NS) & 1), kWaitLimit);
        return;
    }

    // ======================================================= consumers
    const int c0 = blockIdx.y * PG;
    int ncol = nrhs - c0;
    if (ncol > PG) ncol = PG;
    const cplx<T>* pv = Pv + S.coup_off;
    const cplx<T>* ia = inva + S.inva_off;
    cplx<T>* V = buf + tk.buf_off;           // y, then u
    const cplx<T>* B = bsrc + tk.buf_off;    // the local source b
    int prow[RPT];
    bool row[RPT];
    cplx<T> pvp[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        prow[r] = tid + r * NC;
        row[r] = prow[r] < n;
        pvp[r] = row[r] ? pv[prow[r]] : mk<T>(0, 0);
    }
    auto vidx = [&](int c, int j, int pp) -> int64_t {
        return (int64_t)(c0 + c) * rstride + (int64_t)j * n + pp;
    };

    cplx<T> prev[RPT][PG], acc[RPT][PG], pre[RPT][PG];
#pragma unroll
    for (int r = 0; r < RPT; ++r)
#pragma unroll
        for (int c = 0; c < PG; ++c) {
            prev[r][c] = mk<T>(0, 0);
            pre[r][c] = (row[r] && c < ncol) ? B[vidx(c, 0, prow[r])] : mk<T>(0, 0);
        }

    int ci = 0;
    int rb = 0;  // panel buffer of the current line
    auto line_gemv = [&](const cplx<T>* panel) {
#pragma unroll
        for (int r = 0; r < RPT; ++r)
#pragma unroll
            for (int c = 0; c < PG; ++c) acc[r][c] = mk<T>(0, 0);
        for (int k = 0; k < seq.per_line; ++k, ++ci) {
            const int s = ci % NS;
            if (!*abort_flag && !mbar_wait(&full[s], (uint32_t)((ci / NS) & 1), ds.polls)) {
                atomicExch(ds.err, 2);
                *abort_flag = 1;
            }
            const int q0 = seq.col0(ci);
            const int cols = min(cq, n - q0);
            const T* st = stages + s * stage_elems;
#pragma unroll 4
            for (int qq = 0; qq < cols; ++qq) {
                const cplx<T>* rq = panel + (size_t)(q0 + qq) * PG;
                cplx<T> rv[PG];
#pragma unroll
                for (int c = 0; c < PG; ++c) rv[c] = rq[c];
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    const T* Dc = st + (size_t)qq * 2 * nbp + prow[r];
                    const cplx<T> d = row[r] ? mk<T>(Dc[0], Dc[nbp]) : mk<T>(0, 0);
#pragma unroll
                    for (int c = 0; c < PG; ++c) cfma(acc[r][c], d, rv[c]);
                }
            }
            __syncwarp();
            if ((tid & 31) == 0) mbar_arrive(&empty[s]);
        }
    };

    // ---------------- forward: pre holds b_j on entry to line j
    for (int j = 0; j < nl; ++j) {
        cplx<T>* panel = rs + (size_t)rb * nbp_max * PG;
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            if (!row[r]) continue;
            cplx<T> a = (j > 0) ? pvp[r] * ia[j] : mk<T>(0, 0);
#pragma unroll
            for (int c = 0; c < PG; ++c) panel[prow[r] * PG + c] = pre[r][c] - a * prev[r][c];
        }
        if (consumers_sync_any(NC, *abort_flag)) return;
        // prefetch b_{j+1}
#pragma unroll
        for (int r = 0; r < RPT; ++r)
#pragma unroll
            for (int c = 0; c < PG; ++c)
                pre[r][c] = (row[r] && c < ncol && j + 1 < nl) ? B[vidx(c, j + 1, prow[r])]
                                                                : mk<T>(0, 0);
        line_gemv(panel);
#pragma unroll
        for (int r = 0; r < RPT; ++r)
#pragma unroll
            for (int c = 0; c < PG; ++c) {
                prev[r][c] = acc[r][c];
                if (row[r] && c < ncol) V[vidx(c, j, prow[r])] = acc[r][c];
            }
        rb ^= 1;
    }
    // ---------------- backward: prev = u_{j+1}
    for (int j = nl - 2; j >= 0; --j) {
        cplx<T>* panel = rs + (size_t)rb * nbp_max * PG;
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            if (!row[r]) continue;
            cplx<T> cc = pvp[r] * ia[j + 1];
#pragma unroll
            for (int c = 0; c < PG; ++c) panel[prow[r] * PG + c] = cc * prev[r][c];
        }
        if (consumers_sync_any(NC, *abort_flag)) return;
        // y_j, needed after the product
#pragma unroll
        for (int r = 0; r < RPT; ++r)
#pragma unroll
            for (int c = 0; c < PG; ++c)
                pre[r][c] = (row[r] && c < ncol) ? V[vidx(c, j, prow[r])] : mk<T>(0, 0);
        line_gemv(panel);
#pragma unroll
        for (int r = 0; r < RPT; ++r)
#pragma unroll
            for (int c = 0; c < PG; ++c) {
                prev[r][c] = pre[r][c] - acc[r][c];
                if (row[r] && c < ncol) V[vidx(c, j, prow[r])] = prev[r][c];
            }
        rb ^= 1;
    }
}

static SolveGeom geom_for(int nbp_max, size_t esize, int PG, int RPT, size_t* smem) {
    SolveGeom g;
    g.ncons = ((nbp_max + RPT - 1) / RPT + 31) / 32 * 32;
    const size_t col_bytes = 2 * (size_t)nbp_max * esize;
    g.cq = (int)std::max<size_t>(1, (32 * 1024) / col_bytes);
    const size_t rs_bytes = (size_t)2 * nbp_max * PG * 2 * esize;
    const size_t budget = 200 * 1024;
    g.nstage = 6;
    while (g.nstage > 2 && g.nstage * g.cq * col_bytes + rs_bytes + 256 > budget) --g.nstage;
    while (g.nstage * g.cq * col_bytes + rs_bytes + 256 > budget && g.cq > 1) --g.cq;
    *smem = g.nstage * g.cq * col_bytes + rs_bytes + 16 * g.nstage + 16;
    return g;
}

template <typename T, int PG, int RPT>
static void launch_cfg(const Task* tasks, int ntask, const SubDesc* subs, int nbp_max, int nrhs,
                       const T* fac, const cplx<T>* Pv, const cplx<T>* inva, cplx<T>* buf,
                       const cplx<T>* bsrc, int64_t rstride, DevStatus ds, cudaStream_t st) {
    size_t smem = 0;
    SolveGeom g = geom_for(nbp_max, sizeof(T), PG, RPT, &smem);
    cudaFuncSetAttribute(solve_kernel<T, PG, RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    dim3 grid(ntask, (nrhs + PG - 1) / PG);
    solve_kernel<T, PG, RPT><<<grid, g.ncons + 32, smem, st>>>(tasks, subs, nrhs, fac, Pv, inva,
                                                               buf, bsrc, rstride, g, nbp_max, ds);
}

template <typename T, int PG>
static void launch_pg(const Task* tasks, int ntask, const SubDesc* subs, int nbp_max, int nrhs,
                      const T* fac, const cplx<T>* Pv, const cplx<T>* inva, cplx<T>* buf,
                      const cplx<T>* bsrc, int64_t rstride, DevStatus ds, cudaStream_t st) {
    if (nbp_max <= 960)
        launch_cfg<T, PG, 1>(tasks, ntask, subs, nbp_max, nrhs, fac, Pv, inva, buf, bsrc, rstride, ds, st);
    else
        launch_cfg<T, PG, 2>(tasks, ntask, subs, nbp_max, nrhs, fac, Pv, inva, buf, bsrc, rstride, ds, st);
}

template <typename T>
void launch_solve(const Task* tasks, int ntask, const SubDesc* subs, int nbp_max, int nrhs,
                  int panel, const T* fac, const cplx<T>* Pv, const cplx<T>* inva, cplx<T>* buf,
                  const cplx<T>* bsrc, int64_t rstride, DevStatus ds, cudaStream_t st) {
    if (ntask == 0) return;
    switch (panel) {
        case 1: launch_pg<T, 1>(tasks, ntask, subs, nbp_max, nrhs, fac, Pv, inva, buf, bsrc, rstride, ds, st); break;
        case 2: launch_pg<T, 2>(tasks, ntask, subs, nbp_max, nrhs, fac, Pv, inva, buf, bsrc, rstride, ds, st); break;
        case 4: launch_pg<T, 4>(tasks, ntask, subs, nbp_max, nrhs, fac, Pv, inva, buf, bsrc, rstride, ds, st); break;
        default: launch_pg<T, 8>(tasks, ntask, subs, nbp_max, nrhs, fac, Pv, inva, buf, bsrc, rstride, ds, st); break;
    }
}

template void launch_solve<float>(const Task*, int, const SubDesc*, int, int, int, const float*,
                                  const cplx<float>*, const cplx<float>*, cplx<float>*,
                                  const cplx<float>*, int64_t, DevStatus, cudaStream_t);
template void launch_solve<double>(const Task*, int, const SubDesc*, int, int, int,
                                   const double*, const cplx<double>*, const cplx<double>*,
                                   cplx<double>*, const cplx<double>*, int64_t, DevStatus, cudaStream_t);

}  // namespace helm
