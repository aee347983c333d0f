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
// row p of the block for all PG columns.  Per line the right-hand side panel
// (n x PG) sits in shared memory as [q][c]; D_j streams from global memory in
// column-major order, so a warp reads 32 consecutive rows of one column.
// The window buffer holds b on entry, y after the forward pass and u on exit
// (layout [rhs][line][p]).
#include "helm_internal.h"

namespace helm {

template <typename T, int PG>
__global__ void __launch_bounds__(1024) solve_kernel(const Task* __restrict__ tasks,
                                                     const SubDesc* __restrict__ subs, int nrhs,
                                                     const T* __restrict__ fac,
                                                     const cplx<T>* __restrict__ Pv,
                                                     const cplx<T>* __restrict__ inva,
                                                     cplx<T>* buf, int64_t rstride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* rs = reinterpret_cast<cplx<T>*>(smem_raw);  // [nbp][PG]
    const Task tk = tasks[blockIdx.x];
    const SubDesc& S = subs[tk.sub];
    const int n = S.nblk, nbp = S.nbp, nl = S.nlines;
    const int c0 = blockIdx.y * PG;
    const int p = threadIdx.x;
    const bool row = p < n;
    const cplx<T>* pv = Pv + S.coup_off;
    const cplx<T>* ia = inva + S.inva_off;
    const cplx<T> pvp = row ? pv[p] : mk<T>(0, 0);
    cplx<T>* V = buf + tk.buf_off;
    int ncol = nrhs - c0;
    if (ncol > PG) ncol = PG;

    cplx<T> prev[PG], acc[PG];
#pragma unroll
    for (int c = 0; c < PG; ++c) prev[c] = mk<T>(0, 0);

    // ---------------- forward
    for (int j = 0; j < nl; ++j) {
        const T* D = fac + S.fac_off + (int64_t)j * 2 * nbp * nbp;
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
#pragma unroll
        for (int c = 0; c < PG; ++c) acc[c] = mk<T>(0, 0);
        if (row) {
            const T* Dr = D + p;
#pragma unroll 4
            for (int q = 0; q < n; ++q) {
                cplx<T> d = mk<T>(Dr[(int64_t)q * 2 * nbp], Dr[(int64_t)q * 2 * nbp + nbp]);
#pragma unroll
                for (int c = 0; c < PG; ++c) cfma(acc[c], d, rs[q * PG + c]);
            }
#pragma unroll
            for (int c = 0; c < PG; ++c) {
                prev[c] = acc[c];
                if (c < ncol) V[(int64_t)(c0 + c) * rstride + (int64_t)j * n + p] = acc[c];
            }
        }
        __syncthreads();
    }
    // ---------------- backward (prev = u_{L-1} = y_{L-1})
    for (int j = nl - 2; j >= 0; --j) {
        const T* D = fac + S.fac_off + (int64_t)j * 2 * nbp * nbp;
        if (row) {
            cplx<T> cc = pvp * ia[j + 1];
#pragma unroll
            for (int c = 0; c < PG; ++c) rs[p * PG + c] = cc * prev[c];
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < PG; ++c) acc[c] = mk<T>(0, 0);
        if (row) {
            const T* Dr = D + p;
#pragma unroll 4
            for (int q = 0; q < n; ++q) {
                cplx<T> d = mk<T>(Dr[(int64_t)q * 2 * nbp], Dr[(int64_t)q * 2 * nbp + nbp]);
#pragma unroll
                for (int c = 0; c < PG; ++c) cfma(acc[c], d, rs[q * PG + c]);
            }
#pragma unroll
            for (int c = 0; c < PG; ++c) {
                cplx<T> y = (c < ncol) ? V[(int64_t)(c0 + c) * rstride + (int64_t)j * n + p]
                                       : mk<T>(0, 0);
                prev[c] = y - acc[c];
                if (c < ncol) V[(int64_t)(c0 + c) * rstride + (int64_t)j * n + p] = prev[c];
            }
        }
        __syncthreads();
    }
}

template <typename T, int PG>
static void launch_pg(const Task* tasks, int ntask, const SubDesc* subs, int nbp_max, int nrhs,
                      const T* fac, const cplx<T>* Pv, const cplx<T>* inva, cplx<T>* buf,
                      int64_t rstride, cudaStream_t st) {
    size_t smem = sizeof(cplx<T>) * (size_t)nbp_max * PG;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(solve_kernel<T, PG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    dim3 grid(ntask, (nrhs + PG - 1) / PG);
    solve_kernel<T, PG><<<grid, nbp_max, smem, st>>>(tasks, subs, nrhs, fac, Pv, inva, buf,
                                                      rstride);
}

template <typename T>
void launch_solve(const Task* tasks, int ntask, const SubDesc* subs, int nbp_max, int nrhs,
                  int panel, const T* fac, const cplx<T>* Pv, const cplx<T>* inva, cplx<T>* buf,
                  int64_t rstride, cudaStream_t st) {
    if (ntask == 0) return;
    switch (panel) {
        case 1: launch_pg<T, 1>(tasks, ntask, subs, nbp_max, nrhs, fac, Pv, inva, buf, rstride, st); break;
        case 2: launch_pg<T, 2>(tasks, ntask, subs, nbp_max, nrhs, fac, Pv, inva, buf, rstride, st); break;
        case 4: launch_pg<T, 4>(tasks, ntask, subs, nbp_max, nrhs, fac, Pv, inva, buf, rstride, st); break;
        default: launch_pg<T, 8>(tasks, ntask, subs, nbp_max, nrhs, fac, Pv, inva, buf, rstride, st); break;
    }
}

template void launch_solve<float>(const Task*, int, const SubDesc*, int, int, int, const float*,
                                  const cplx<float>*, const cplx<float>*, cplx<float>*, int64_t,
                                  cudaStream_t);
template void launch_solve<double>(const Task*, int, const SubDesc*, int, int, int,
                                   const double*, const cplx<double>*, const cplx<double>*,
                                   cplx<double>*, int64_t, cudaStream_t);

}  // namespace helm
