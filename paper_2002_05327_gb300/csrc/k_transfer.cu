// Local sources, source transfer and assembly of Algorithm 3.1 / 4.1.
//
// gather: for every (sweep l, subdomain) solve of a dependency level, write its
// local source on the whole window:
//     r^l = [l = 1] J f chi_{Omega_ij}  +  sum over incoming (dir, l_src) of
//           J_recv Psi_{dir; sender}(u^{l_src}_sender),
//     J_recv Psi_{dir; I}(v) = -A_recv(beta_{dir; I} v) chi_{dir; I}
// (Section 2.2; Algorithm 3.1 "add the transferred source to the l'-th local
// source of the neighbour").  Each window node is summed by one thread in a
// fixed order of the incoming list, so the result is deterministic without
// atomics.  The transfer is non-zero only on the strip beyond the sender's box
// face(s): nodes m = 0..d beyond each face (beta = beta_hat(m/d) vanishes from
// m = d on, and its residual reaches one node further).
//
// assemble: u_DDM = sum_l sum_ij beta_{0,0;ij} u^l_ij (Eq. 3.x / 4.x), summed
// per global node over the at most 2^n boxes whose cutoff reaches it.
#include <type_traits>

#include "helm_internal.h"
#include "ff.h"

namespace helm {

// beta^{(a)}_{dir, box}(k): beta_hat(m/d) at the m-th node beyond the face the
// direction points through, 1 elsewhere (tab[m] = beta_hat(m/d), tab[d] = 0).
template <typename T>
__device__ __forceinline__ T beta1(int dir, int k, int blo, int bhi, int d, const T* tab) {
    if (dir > 0 && k >= bhi) return tab[min(k - bhi, d)];
    if (dir < 0 && k < blo) return tab[min(blo - 1 - k, d)];
    return T(1);
}

constexpr int kMaxIncoming = 32;  // routing gives at most 8 (2D) / 26 (3D); the host checks
constexpr int kRG = 8;             // right-hand sides per thread

// an entry of the global source (complex128, or float-float for the Krylov
// work vectors) in the window precision, off the FP64 pipe for complex64
template <typename T>
__device__ __forceinline__ cplx<T> src_cast(cplx<double> v) {
    if constexpr (sizeof(T) == 4)
        return mk<float>(ffa::d2f(v.re), ffa::d2f(v.im));
    else
        return v;
}
template <typename T>
__device__ __forceinline__ cplx<T> src_cast(float4 v) {
    if constexpr (sizeof(T) == 4)
        return mk<float>(v.x + v.y, v.z + v.w);
    else
        return mk<double>(ffa::join_d({v.x, v.y}), ffa::join_d({v.z, v.w}));
}

// Block = up to kGB consecutive nodes of one task's work list (GNode: the
// window nodes the first sweep's box or an incoming strip reaches, with the
// incoming transfers that reach each), so every thread has a node to write.
// The task's incoming transfers are staged in shared memory; each thread
// handles kRG right-hand sides with independent loads and sums the transfers
// in the order of the incoming list.
template <typename T, typename VB>
__global__ void __launch_bounds__(kGB) gather_kernel(const GBlock* __restrict__ blocks,
                                                     const GNode* __restrict__ nodes,
                                                     const Task* __restrict__ tasks,
                                                     const SubDesc* __restrict__ subs,
                                                     const Incoming* __restrict__ inc, DevProblem P, T ih2,
                                                     T omega2, const T* __restrict__ m,
                                                     const cplx<T>* __restrict__ an,
                                                     const cplx<T>* __restrict__ af,
                                                     const T* __restrict__ tab,
                                                     const VB* __restrict__ b, int nrhs,
                                                     const cplx<T>* __restrict__ buf, cplx<T>* bsrc,
                                                     int64_t rstride) {
    struct InS {
        int dir[3];
        int blo[3], bhi[3];  // sender box
        int lo[3], nw[3];    // sender window
        int64_t off;         // sender buffer offset
    };
    __shared__ InS sin[kMaxIncoming];
    __shared__ T stab[129];
    const GBlock gb = blocks[blockIdx.x];
    const bool act = (int)threadIdx.x < gb.cnt;
    const GNode nd = act ? nodes[gb.node0 + threadIdx.x] : GNode{0u, 0u};
    const Task tk = tasks[gb.task];
    const SubDesc& S = subs[tk.sub];
    const int ni = tk.in_cnt;
    if ((int)threadIdx.x < ni) {
        const int i = threadIdx.x;
        const Incoming I = inc[tk.in_off + i];
        const SubDesc& R = subs[I.sender];
        for (int a = 0; a < 3; ++a) {
            sin[i].dir[a] = I.dir[a];
            sin[i].blo[a] = R.box_lo[a];
            sin[i].bhi[a] = R.box_hi[a];
            sin[i].lo[a] = R.lo[a];
            sin[i].nw[a] = R.nw[a];
        }
        sin[i].off = I.sender_buf_off;
    }
    for (int i = threadIdx.x; i <= P.d; i += blockDim.x) stab[i] = tab[i];
    __syncthreads();
    if (!act) return;
    const int ndim = P.ndim;
    const int64_t k = nd.k;
    int x[3];
    x[0] = (int)(k % S.nw[0]);
    x[1] = (int)((k / S.nw[0]) % S.nw[1]);
    x[2] = (int)(k / ((int64_t)S.nw[0] * S.nw[1]));
    int g[3];
    for (int a = 0; a < 3; ++a) g[a] = S.lo[a] + x[a];
    const int64_t Ng = (int64_t)P.N[0] * P.N[1] * P.N[2];
    const int64_t gidx = ((int64_t)g[2] * P.N[1] + g[1]) * P.N[0] + g[0];
    const int c0 = blockIdx.y * kRG;
    const int nc = min(kRG, nrhs - c0);
    cplx<T>* __restrict__ out = bsrc + tk.buf_off + k + (int64_t)c0 * rstride;
    const cplx<T>* __restrict__ src = buf;  // sender solutions

    const bool inbox = (nd.mask >> 31) != 0u;
    cplx<T> val[kRG];
#pragma unroll
    for (int c = 0; c < kRG; ++c)
        val[c] = (inbox && c < nc) ? src_cast<T>(b[(int64_t)(c0 + c) * Ng + gidx]) : mk<T>(0, 0);

    unsigned int todo = nd.mask & 0x7FFFFFFFu;
    if (todo) {
        Win<T> w;
        for (int a = 0; a < 3; ++a) {
            w.lo[a] = S.lo[a];
            w.n[a] = S.nw[a];
            w.alpha_node[a] = an + S.alpha_off[a];
            w.alpha_face[a] = af + S.face_off[a];
        }
        const Stencil<T> st = stencil_at(w, ndim, x, ih2, omega2, m[gidx]);
        cplx<T> coef[7];
        coef[0] = st.diag;
        for (int a = 0; a < 3; ++a) {
            coef[1 + 2 * a] = st.cp[a];
            coef[2 + 2 * a] = st.cm[a];
        }
        const int npt = 1 + 2 * ndim;
        while (todo) {  // incoming transfers reaching this node, in list order
            const InS& R = sin[__ffs(todo) - 1];
            todo &= todo - 1;
            // stencil points (static indices after unrolling: the arrays stay in registers)
#pragma unroll
            for (int pt = 0; pt < 7; ++pt) {
                if (pt >= npt) break;
                int gg[3] = {g[0], g[1], g[2]};
                bool ok = true;
                if (pt > 0) {
                    const int ax = (pt - 1) / 2, o = (pt & 1) ? 1 : -1;
                    gg[ax] += o;
                    const int xl = gg[ax] - S.lo[ax];
                    ok = xl >= 0 && xl < S.nw[ax];  // Dirichlet outside the receiver window
                }
                T beta = T(1);
                int64_t li = 0;
#pragma unroll
                for (int a = 2; a >= 0; --a) {
                    if (a >= ndim || !ok) continue;
                    const int xl = gg[a] - R.lo[a];
                    if (xl < 0 || xl >= R.nw[a]) ok = false;  // zero outside the sender window
                    li = li * R.nw[a] + xl;
                    const int dd = R.dir[a];
                    if (dd > 0 && gg[a] >= R.bhi[a]) beta *= stab[min(gg[a] - R.bhi[a], P.d)];
                    if (dd < 0 && gg[a] < R.blo[a]) beta *= stab[min(R.blo[a] - 1 - gg[a], P.d)];
                }
                if (!ok || beta == T(0)) continue;
                const cplx<T> cw = beta * coef[pt];
                const cplx<T>* sp = src + R.off + li + (int64_t)c0 * rstride;
#pragma unroll
                for (int c = 0; c < kRG; ++c)
                    if (c < nc) val[c] = val[c] - cw * sp[(int64_t)c * rstride];
            }
        }
    }
#pragma unroll
    for (int c = 0; c < kRG; ++c)
        if (c < nc) out[(int64_t)c * rstride] = val[c];
}

template <typename T, typename VB>
void launch_gather(const GBlock* blocks, int nblocks, const GNode* nodes, const Task* tasks,
                   const SubDesc* subs, const Incoming* inc, const DevProblem& P, const T* m,
                   const cplx<T>* an, const cplx<T>* af, const T* beta_tab, const VB* b, int nrhs,
                   const cplx<T>* buf, cplx<T>* bsrc, int64_t rstride, cudaStream_t st) {
    if (nblocks == 0) return;
    dim3 grid((unsigned)nblocks, (nrhs + kRG - 1) / kRG);
    gather_kernel<T, VB><<<grid, kGB, 0, st>>>(blocks, nodes, tasks, subs, inc, P, T(1.0 / (P.h * P.h)),
                                           T(P.omega * P.omega), m, an, af, beta_tab, b, nrhs, buf, bsrc,
                                           rstride);
}

// ----------------------------------------------------------------------------- assembly
constexpr int kAG = 8;  // right-hand sides per assembly thread
// sweeps whose loads a thread issues together (complex64 windows; complex128
// ones take one at a time, as their sums already fill the registers)
template <typename T>
constexpr int assemble_sweeps() { return sizeof(T) == 4 ? 2 : 1; }

template <int NDIM, typename T, typename VU>
__global__ void __launch_bounds__(256, 2)
    assemble_kernel(DevProblem P, const SubDesc* __restrict__ subs, const int* __restrict__ box_of,
                    const int64_t* __restrict__ node_buf, int nsweeps, const T* __restrict__ tab,
                    const cplx<T>* __restrict__ buf, int64_t rstride, int nrhs, VU* U) {
    // one thread per (global node, group of kAG right-hand sides): the boxes
    // whose cutoff reaches the node and their weights are found once, then
    // applied to the group, the loads of kASW sweeps issued together
    constexpr int kASW = assemble_sweeps<T>();
    const int64_t Ng = (int64_t)P.N[0] * P.N[1] * P.N[2];
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Ng) return;
    const int c0 = blockIdx.y * kAG;
    int g[3] = {0, 0, 0};
    if (Ng <= (int64_t)UINT32_MAX) {  // 32-bit index arithmetic (uniform over the launch)
        const uint32_t kk = (uint32_t)k, n0 = (uint32_t)P.N[0], q = kk / n0;
        g[0] = (int)(kk - q * n0);
        if (NDIM == 2) {
            g[1] = (int)q;
        } else {
            const uint32_t n1 = (uint32_t)P.N[1], q2 = q / n1;
            g[1] = (int)(q - q2 * n1);
            g[2] = (int)q2;
        }
    } else {
        g[0] = (int)(k % P.N[0]);
        g[1] = (int)((k / P.N[0]) % P.N[1]);
        g[2] = (int)(k / ((int64_t)P.N[0] * P.N[1]));
    }
    // candidate boxes per axis in fixed slots: 0 the own box (cutoff 1), 1 the
    // box above and 2 the box below, each with the weight of its cutoff at this
    // node (0 where its cutoff does not reach)
    int cb[NDIM][3];
    T cw[NDIM][3];
    int off = 0;
#pragma unroll
    for (int a = 0; a < NDIM; ++a) {
        cb[a][1] = cb[a][2] = 0;
        cw[a][0] = T(1);
        cw[a][1] = cw[a][2] = T(0);
        const int i0 = box_of[off + g[a]];
        off += P.N[a];
        cb[a][0] = i0;
        int stride = 1;
        for (int b2 = 0; b2 < a; ++b2) stride *= P.nb[b2];
        // neighbour above: its lower cutoff at the m-th node below its face
        if (i0 + 1 < P.nb[a]) {
            const int lo1 = subs[(i0 + 1) * stride].box_lo[a];
            const int mm = lo1 - 1 - g[a];
            if (mm < P.d) {
                cb[a][1] = i0 + 1;
                cw[a][1] = tab[mm];
            }
        }
        if (i0 > 0) {
            const int hi0 = subs[(i0 - 1) * stride].box_hi[a];
            const int mm = g[a] - hi0;
            if (mm < P.d) {
                cb[a][2] = i0 - 1;
                cw[a][2] = tab[mm];
            }
        }
    }
    // boxes with a non-zero weight, in a fixed order: (window offset of the
    // node, weight).  Where every box is at least 2d wide, at most 2^NDIM
    // boxes reach a node; narrower boxes (down to d + 2) let both neighbours
    // of an axis reach it: 9 in 2D, all kept; in 3D the first 8 are kept
    constexpr int kMaxBox = NDIM == 2 ? 9 : 8;
    int sb[kMaxBox];
    int lib[kMaxBox];  // window offsets (a window holds fewer than 2^31 nodes)
    T wb[kMaxBox];
    int nbx = 0;
#pragma unroll
    for (int ib = 0; ib < kMaxBox; ++ib) {
        sb[ib] = 0;
        lib[ib] = 0;
        wb[ib] = T(0);
    }
#pragma unroll
    for (int i0 = 0; i0 < 3; ++i0)
#pragma unroll
        for (int i1 = 0; i1 < 3; ++i1)
#pragma unroll
            for (int i2 = 0; i2 < (NDIM == 3 ? 3 : 1); ++i2) {
                const T wgt = NDIM == 3 ? cw[0][i0] * cw[1][i1] * cw[NDIM - 1][i2] : cw[0][i0] * cw[1][i1] * T(1);
                if (wgt == T(0) || nbx >= kMaxBox) continue;
                const int s = cb[0][i0] + P.nb[0] * (cb[1][i1] + (NDIM == 3 ? P.nb[1] * cb[NDIM - 1][i2] : 0));
                const SubDesc& S = subs[s];
                int li = 0;
#pragma unroll
                for (int a = NDIM - 1; a >= 0; --a) li = li * S.nw[a] + (g[a] - S.lo[a]);
#pragma unroll
                for (int ib = 0; ib < kMaxBox; ++ib)  // register-resident list: static indices
                    if (ib == nbx) {
                        sb[ib] = s;
                        lib[ib] = li;
                        wb[ib] = wgt;
                    }
                ++nbx;
            }
    // complex64 windows: float-float sums (no FP64 instruction per term);
    // complex128 windows: doubles
    constexpr bool kF32 = sizeof(T) == 4;
    double sr[kAG], si[kAG];
    ffa::ff fr[kAG], fi[kAG];
#pragma unroll
    for (int c = 0; c < kAG; ++c) {
        sr[c] = si[c] = 0;
        fr[c] = fi[c] = ffa::ff{0.f, 0.f};
    }
#pragma unroll
    for (int ib = 0; ib < kMaxBox; ++ib) {
        if (ib >= nbx) break;
        for (int l0 = 0; l0 < nsweeps; l0 += kASW) {
            // the loads of kASW sweeps first, then the sums in sweep order
            int64_t ob[kASW];
            cplx<T> v[kASW][kAG];
#pragma unroll
            for (int q = 0; q < kASW; ++q) {
                ob[q] = l0 + q < nsweeps ? node_buf[(int64_t)(l0 + q) * P.nsub + sb[ib]] : -1;
                const cplx<T>* bp = buf + (ob[q] < 0 ? 0 : ob[q] + (int64_t)lib[ib] + (int64_t)c0 * rstride);
#pragma unroll
                for (int c = 0; c < kAG; ++c)
                    v[q][c] = (ob[q] >= 0 && c0 + c < nrhs) ? bp[(int64_t)c * rstride] : mk<T>(0, 0);
            }
#pragma unroll
            for (int q = 0; q < kASW; ++q) {
                if (ob[q] < 0) continue;
#pragma unroll
                for (int c = 0; c < kAG; ++c) {
                    if constexpr (kF32) {
                        ffa::acc_add(fr[c], wb[ib] * v[q][c].re);
                        ffa::acc_add(fi[c], wb[ib] * v[q][c].im);
                    } else {
                        sr[c] += wb[ib] * v[q][c].re;
                        si[c] += wb[ib] * v[q][c].im;
                    }
                }
            }
        }
    }
#pragma unroll
    for (int c = 0; c < kAG; ++c) {
        if (c0 + c >= nrhs) continue;
        if constexpr (!kF32 && std::is_same<VU, cplx<double>>::value) {
            U[(int64_t)(c0 + c) * Ng + k] = mk<double>(sr[c], si[c]);
        } else {
            if constexpr (!kF32) {
                fr[c] = ffa::split_d(sr[c]);
                fi[c] = ffa::split_d(si[c]);
            }
            ffa::st_c(U + (int64_t)(c0 + c) * Ng + k, ffa::cff{fr[c], fi[c]});
        }
    }
}

template <typename T, typename VU>
void launch_assemble(const DevProblem& P, const SubDesc* subs, const int* box_of,
                     const int64_t* node_buf, int nsweeps, const T* beta_tab,
                     const cplx<T>* buf, int64_t rstride, int nrhs, VU* U, cudaStream_t st) {
    const int64_t Ng = (int64_t)P.N[0] * P.N[1] * P.N[2];
    const int nt = 256;
    dim3 grid((unsigned)((Ng + nt - 1) / nt), (nrhs + kAG - 1) / kAG);
    if (P.ndim == 2)
        assemble_kernel<2, T, VU><<<grid, nt, 0, st>>>(P, subs, box_of, node_buf, nsweeps, beta_tab, buf, rstride,
                                                       nrhs, U);
    else
        assemble_kernel<3, T, VU><<<grid, nt, 0, st>>>(P, subs, box_of, node_buf, nsweeps, beta_tab, buf, rstride,
                                                       nrhs, U);
}

#define HELM_TRANSFER_INST(T, V)                                                                          \
    template void launch_gather<T, V>(const GBlock*, int, const GNode*, const Task*, const SubDesc*,           \
                                      const Incoming*, const DevProblem&, const T*, const cplx<T>*,            \
                                      const cplx<T>*, const T*, const V*, int, const cplx<T>*, cplx<T>*,       \
                                      int64_t, cudaStream_t);                                                  \
    template void launch_assemble<T, V>(const DevProblem&, const SubDesc*, const int*, const int64_t*, int,    \
                                        const T*, const cplx<T>*, int64_t, int, V*, cudaStream_t);
HELM_TRANSFER_INST(float, cplx<double>)
HELM_TRANSFER_INST(float, float4)
HELM_TRANSFER_INST(double, cplx<double>)
HELM_TRANSFER_INST(double, float4)
#undef HELM_TRANSFER_INST

}  // namespace helm
