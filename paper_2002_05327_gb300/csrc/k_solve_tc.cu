// Subdomain solves on the tensor cores (precision HELM_PREC_TF32).
//
// Same recurrence as k_solve.cu (block-Thomas forward y_j = D_j(b_j - a_j y_{j-1}),
// backward u_j = y_j - D_j(c_j u_{j+1})), with each block product D_j R done
// as one real GEMM on the tensor cores, TF32 inputs and FP32 accumulation:
//
//   K index k = 2q + part  (q: block column, part 0 = Re D, 1 = Im D)
//   A[p][2q+part]  = part ? Im D(p,q) : Re D(p,q)       (the stored block, as is)
//   N index n = 2c + w     (c: right-hand side, w 0 = Re y, 1 = Im y)
//   B[2q][2c] = Re r_qc   B[2q+1][2c] = -Im r_qc   B[2q][2c+1] = Im r_qc   B[2q+1][2c+1] = Re r_qc
//
// so that (A B)[p][2c] = Re y_pc and (A B)[p][2c+1] = Im y_pc.  With the
// m16n8k8 accumulator layout, lane (g, t) of a warp holds columns 2t, 2t+1 of
// rows g and g+8: exactly (Re, Im) of right-hand side t -- every thread owns
// whole complex outputs and builds the next line's B rows for them.
//
// A comes straight from the column-major factor storage: the producer warp
// bulk-copies whole column spans into a ring of shared stages (full/empty
// mbarriers, bounded waits), as in k_solve.cu.  The padded block size
// nbp = 8 (mod 32) puts the four planes an A fragment touches (columns q,q+1,
// Re/Im) in disjoint banks; B lives in shared memory as [k][n] with a row
// stride that keeps the B fragment loads conflict-free too.  One named barrier
// per line step among the consumer warps; B is double-buffered.
#include <algorithm>

#include "helm_internal.h"

namespace helm {

namespace {

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
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr uint32_t kWaitLimit = kDrainPolls;

}  // namespace

struct TcGeom {
    int cq;      // block columns per chunk (multiple of 4)
    int nstage;  // ring depth
    int ncw;     // consumer warps
    int kpad;    // B rows = 2 * kpad, kpad >= every roundup4(n)
};

template <int NT, int MTW>
__global__ void __launch_bounds__(1024) solve_tc_kernel(const Task* __restrict__ tasks,
                                                        const SubDesc* __restrict__ subs,
                                                        int nrhs, const float* __restrict__ fac,
                                                        const cplx<float>* __restrict__ Pv,
                                                        const cplx<float>* __restrict__ inva,
                                                        cplx<float>* buf,
                                                        const cplx<float>* __restrict__ bsrc,
                                                        int64_t rstride,
                                                        TcGeom G, int nbp_max, DevStatus ds) {
    constexpr int PG = 4 * NT;
    constexpr int BS = 8 * NT + (NT > 1 ? 8 : 0);  // floats per B row
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const Task tk = tasks[blockIdx.x];
    const SubDesc& S = subs[tk.sub];
    const int n = S.nblk, nbp = S.nbp, nl = S.nlines;
    const int n4 = (n + 3) & ~3;
    const int cq = G.cq, NS = G.nstage, NCW = G.ncw, NC = 32 * NCW;
    const size_t stage_elems = (size_t)cq * 2 * nbp_max;
    const size_t bmat_elems = (size_t)2 * G.kpad * BS;
    float* stages = reinterpret_cast<float*>(smem_raw);
    float* bmat = stages + stage_elems * NS;  // [2][2*kpad][BS]
    uint64_t* full = reinterpret_cast<uint64_t*>(bmat + 2 * bmat_elems);
    uint64_t* empty = full + NS;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + NS);

    const int per_line = (n4 + cq - 1) / cq;
    const int total = (2 * nl - 1) * per_line;
    const int tid = threadIdx.x;
    if (tid == 0) {
        *abort_flag = 0;
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (size_t i = tid; i < 2 * bmat_elems; i += blockDim.x) bmat[i] = 0.f;
    __syncthreads();

    // ======================================================= producer warp
    if (tid >= NC) {
        if (tid != NC) return;
        const float* fbase = fac + S.fac_off;
        const size_t line_elems = (size_t)2 * nbp * nbp;
        int issued = 0;
        for (int i = 0; i < total; ++i) {
            const int s = i % NS;
            if (i >= NS && !mbar_wait(&empty[s], (uint32_t)(((i / NS) - 1) & 1), ds.polls)) {
                atomicExch(ds.err, 2);
                *abort_flag = 1;
            }
            if (*abort_flag) break;
            const int li = i / per_line;
            const int l = li < nl ? li : 2 * nl - 2 - li;
            const int q0 = (i % per_line) * cq;
            const int cols = min(cq, n4 - q0);
            const uint32_t bytes = (uint32_t)(cols * 2 * nbp * sizeof(float));
            mbar_expect_tx(&full[s], bytes);
            bulk_g2s(stages + s * stage_elems, fbase + l * line_elems + (size_t)q0 * 2 * nbp, bytes,
                     &full[s]);
            issued = i + 1;
        }
        for (int i = max(0, issued - NS); i < issued; ++i)
            mbar_wait(&full[i % NS], (uint32_t)((i / NS) & 1), kWaitLimit);
        return;
    }

    // ======================================================= consumers
    const int warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    const int c0 = blockIdx.y * PG;
    const cplx<float>* pv = Pv + S.coup_off;
    const cplx<float>* ia = inva + S.inva_off;
    cplx<float>* V = buf + tk.buf_off;          // y, then u
    const cplx<float>* B = bsrc + tk.buf_off;   // the local source b

    // owned outputs: rows row[i][h] = 16*(warp*MTW+i) + g + 8h, columns c = 4*nt + t
    int row[MTW][2];
    bool rv[MTW][2];
    cplx<float> pvr[MTW][2];
    bool cv[NT];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) cv[nt] = c0 + 4 * nt + t < nrhs;
#pragma unroll
    for (int i = 0; i < MTW; ++i)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            row[i][h] = 16 * (warp * MTW + i) + g + 8 * h;
            rv[i][h] = row[i][h] < n;
            pvr[i][h] = rv[i][h] ? pv[row[i][h]] : mk<float>(0, 0);
        }
    auto vidx = [&](int nt, int j, int r) -> int64_t {
        return (int64_t)(c0 + 4 * nt + t) * rstride + (int64_t)j * n + r;
    };
    // write r_{q=r, c} into B rows 2r, 2r+1 of buffer bb
    auto put_b = [&](int bb, int r, int nt, cplx<float> v) {
        float* B0 = bmat + bb * bmat_elems + (size_t)(2 * r) * BS + 8 * nt + 2 * t;
        B0[0] = __uint_as_float(to_tf32(v.re));
        B0[1] = __uint_as_float(to_tf32(v.im));
        B0[BS] = __uint_as_float(to_tf32(-v.im));
        B0[BS + 1] = __uint_as_float(to_tf32(v.re));
    };

    cplx<float> prev[MTW][2][NT], pre[MTW][2][NT];
    float acc[MTW][NT][4];
    // line 0 panel: r_0 = b_0
#pragma unroll
    for (int i = 0; i < MTW; ++i)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                cplx<float> b = (rv[i][h] && cv[nt]) ? B[vidx(nt, 0, row[i][h])] : mk<float>(0, 0);
                prev[i][h][nt] = mk<float>(0, 0);
                if (row[i][h] < n4) put_b(0, row[i][h], nt, b);
            }

    int ci = 0;
    const int nsteps = 2 * nl - 1;
    for (int step = 0; step < nsteps; ++step) {
        const bool fwd = step < nl;
        const int j = fwd ? step : 2 * nl - 2 - step;
        const int bb = step & 1;
        if (consumers_sync_any(NC, *abort_flag)) return;
        // operands needed after the product: b_{j+1} (forward) or y_j (backward)
#pragma unroll
        for (int i = 0; i < MTW; ++i)
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    const int jj = fwd ? j + 1 : j;
                    const bool ld = rv[i][h] && cv[nt] && jj < nl;
                    pre[i][h][nt] = ld ? (fwd ? B : V)[vidx(nt, jj, row[i][h])] : mk<float>(0, 0);
                }
#pragma unroll
        for (int i = 0; i < MTW; ++i)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[i][nt][e] = 0.f;
        const float* Bc = bmat + bb * bmat_elems;
        for (int k = 0; k < per_line; ++k, ++ci) {
            const int s = ci % NS;
            if (!*abort_flag && !mbar_wait(&full[s], (uint32_t)((ci / NS) & 1), ds.polls)) {
                atomicExch(ds.err, 2);
                *abort_flag = 1;
            }
            const int q0 = k * cq;
            const int ksteps = min(cq, n4 - q0) >> 2;
            const float* st = stages + s * stage_elems;
            for (int ks = 0; ks < ksteps; ++ks) {
                // k' = 8ks + t -> column qa = 4ks + t/2, plane t&1; k' + 4 -> column qa + 2
                const int qa = 4 * ks + (t >> 1);
                const float* A0 = st + (size_t)qa * 2 * nbp + (t & 1) * nbp;
                const float* A1 = A0 + 4 * nbp;
                uint32_t a[MTW][4];
#pragma unroll
                for (int i = 0; i < MTW; ++i) {
                    const int m0 = 16 * (warp * MTW + i) + g;
                    a[i][0] = __float_as_uint(A0[m0]);
                    a[i][1] = __float_as_uint(A0[m0 + 8]);
                    a[i][2] = __float_as_uint(A1[m0]);
                    a[i][3] = __float_as_uint(A1[m0 + 8]);
                }
                const int kb = 2 * (q0 + 4 * ks) + t;  // B row of b0 (b1: +4)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    const uint32_t b0 = __float_as_uint(Bc[(size_t)kb * BS + 8 * nt + g]);
                    const uint32_t b1 = __float_as_uint(Bc[(size_t)(kb + 4) * BS + 8 * nt + g]);
#pragma unroll
                    for (int i = 0; i < MTW; ++i) mma_tf32(acc[i][nt], a[i], b0, b1);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
        // epilogue: outputs, then the B rows of the next step
        const int nbb = bb ^ 1;
#pragma unroll
        for (int i = 0; i < MTW; ++i)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = row[i][h];
                cplx<float> coup = mk<float>(0, 0);
                if (rv[i][h]) {
                    if (fwd && j + 1 < nl) coup = pvr[i][h] * ia[j + 1];       // a_{j+1}
                    else if (fwd) coup = pvr[i][h] * ia[nl - 1];                // c_{nl-2}
                    else if (j > 0) coup = pvr[i][h] * ia[j];                   // c_{j-1}
                }
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    const cplx<float> y = mk<float>(acc[i][nt][2 * h], acc[i][nt][2 * h + 1]);
                    cplx<float> out;
                    if (fwd) out = y;
                    else out = pre[i][h][nt] - y;
                    if (rv[i][h] && cv[nt]) V[vidx(nt, j, r)] = out;
                    prev[i][h][nt] = out;
                    cplx<float> nb = mk<float>(0, 0);
                    if (rv[i][h]) {
                        if (fwd && j + 1 < nl) nb = pre[i][h][nt] - coup * out;  // r_{j+1}
                        else nb = coup * out;                                      // c (*) u
                    }
                    if (step + 1 < nsteps && r < n4) put_b(nbb, r, nt, nb);
                }
            }
    }
}

static TcGeom tc_geom(int nbp_max, int kpad, int mtiles, int MTW, int NT, size_t* smem) {
    TcGeom G;
    G.ncw = (mtiles + MTW - 1) / MTW;
    G.kpad = kpad;
    const size_t col_bytes = 2 * (size_t)nbp_max * sizeof(float);
    const int BS = 8 * NT + (NT > 1 ? 8 : 0);
    const size_t bmat_bytes = (size_t)2 * 2 * kpad * BS * sizeof(float);
    G.cq = std::max<int>(4, (int)((24 * 1024) / col_bytes) & ~3);
    // as many bytes in flight as shared memory allows: the block stream is
    // latency-bound per SM, so its rate grows with the depth of the ring
    const size_t budget = 220 * 1024;
    G.nstage = 12;
    while (G.nstage > 2 && G.nstage * G.cq * col_bytes + bmat_bytes + 256 > budget) --G.nstage;
    while (G.nstage * G.cq * col_bytes + bmat_bytes + 256 > budget && G.cq > 4) G.cq -= 4;
    *smem = G.nstage * G.cq * col_bytes + bmat_bytes + 16 * G.nstage + 16;
    return G;
}

template <int NT, int MTW>
static void launch_tc(const Task* tasks, int ntask, const SubDesc* subs, int nbp_max, int nrhs,
                      const float* fac, const cplx<float>* Pv, const cplx<float>* inva,
                      cplx<float>* buf, const cplx<float>* bsrc, int64_t rstride, DevStatus ds,
                      cudaStream_t st) {
    const int mtiles = (nbp_max + 15) / 16;
    const int kpad = ((nbp_max + 3) & ~3);
    size_t smem = 0;
    TcGeom G = tc_geom(nbp_max, kpad, mtiles, MTW, NT, &smem);
    cudaFuncSetAttribute(solve_tc_kernel<NT, MTW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    dim3 grid(ntask, (nrhs + 4 * NT - 1) / (4 * NT));
    solve_tc_kernel<NT, MTW><<<grid, 32 * G.ncw + 32, smem, st>>>(tasks, subs, nrhs, fac, Pv,
                                                                  inva, buf, bsrc, rstride, G, nbp_max,
                                                                  ds);
}

void launch_solve_tc(const Task* tasks, int ntask, const SubDesc* subs, int nbp_max, int nrhs,
                     int panel, const float* fac, const cplx<float>* Pv, const cplx<float>* inva,
                     cplx<float>* buf, const cplx<float>* bsrc, int64_t rstride, DevStatus ds,
                     cudaStream_t st) {
    if (ntask == 0) return;
    const int mtiles = (nbp_max + 15) / 16;
    const int MTW = mtiles <= 31 ? 1 : mtiles <= 62 ? 2 : 4;
    const bool wide = panel >= 8;
#define HELM_TC(NT_, MTW_) \
    launch_tc<NT_, MTW_>(tasks, ntask, subs, nbp_max, nrhs, fac, Pv, inva, buf, bsrc, rstride, ds, st)
    if (MTW == 1) {
        if (panel >= 16) HELM_TC(4, 1); else if (wide) HELM_TC(2, 1); else HELM_TC(1, 1);
    } else if (MTW == 2) {
        if (wide) HELM_TC(2, 2); else HELM_TC(1, 2);
    } else {
        HELM_TC(1, 4);
    }
#undef HELM_TC
}

// Round a factor array to TF32 in place (round to nearest, ties away).
__global__ void round_tf32_kernel(float* x, int64_t count) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) x[i] = __uint_as_float(to_tf32(x[i]));
}

void launch_round_tf32(float* x, int64_t count, cudaStream_t st) {
    round_tf32_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(x, count);
}

}  // namespace helm
