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
#include "helm_internal.h"

namespace helm {

// beta^{(a)}_{dir, box}(k): beta_hat(m/d) at the m-th node beyond the face the
// direction points through, 1 elsewhere (tab[m] = beta_hat(m/d), tab[d] = 0).
template <typename T>
__device__ __forceinline__ T beta1(int dir, int k, int blo, int bhi, int d, const T* tab) {
    if (dir > 0 && k >= bhi) return tab[min(k - bhi, d)];
    if (dir < 0 && k < blo) return tab[min(blo - 1 - k, d)];
    return T(1);
}

template <typename T>
__global__ void gather_kernel(const Task* __restrict__ tasks, const SubDesc* __restrict__ subs,
                              const Incoming* __restrict__ inc, DevProblem P,
                              const T* __restrict__ m, const cplx<T>* __restrict__ an,
                              const cplx<T>* __restrict__ af, const T* __restrict__ tab,
                              const cplx<double>* __restrict__ b, int nrhs, cplx<T>* buf,
                              int64_t rstride) {
    const Task tk = tasks[blockIdx.y];
    const SubDesc& S = subs[tk.sub];
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.z;
    if (k >= S.win_elems) return;
    const int ndim = P.ndim;
    int x[3];
    x[0] = (int)(k % S.nw[0]);
    x[1] = (int)((k / S.nw[0]) % S.nw[1]);
    x[2] = (int)(k / ((int64_t)S.nw[0] * S.nw[1]));
    int g[3];
    for (int a = 0; a < 3; ++a) g[a] = S.lo[a] + x[a];
    const int64_t Ng = (int64_t)P.N[0] * P.N[1] * P.N[2];
    const int64_t gidx = ((int64_t)g[2] * P.N[1] + g[1]) * P.N[0] + g[0];

    cplx<T> val = mk<T>(0, 0);
    if (tk.sweep == 0) {
        bool inbox = true;
        for (int a = 0; a < ndim; ++a) inbox &= (g[a] >= S.box_lo[a]) && (g[a] < S.box_hi[a]);
        if (inbox) val = ccast<T>(b[(int64_t)c * Ng + gidx]);
    }
    if (tk.in_cnt > 0) {
        Win<T> w;
        for (int a = 0; a < 3; ++a) {
            w.lo[a] = S.lo[a];
            w.n[a] = S.nw[a];
            w.alpha_node[a] = an + S.alpha_off[a];
            w.alpha_face[a] = af + S.face_off[a];
        }
        bool have_st = false;
        Stencil<T> st;
        for (int i = 0; i < tk.in_cnt; ++i) {
            const Incoming I = inc[tk.in_off + i];
            const SubDesc& R = subs[I.sender];
            bool in = true;
            for (int a = 0; a < ndim; ++a) {
                if (I.dir[a] > 0) in &= (g[a] >= R.box_hi[a]) && (g[a] <= R.box_hi[a] + P.d);
                if (I.dir[a] < 0) in &= (g[a] < R.box_lo[a]) && (g[a] >= R.box_lo[a] - 1 - P.d);
            }
            if (!in) continue;
            if (!have_st) {
                T mv = m[gidx];
                st = stencil_at(w, ndim, x, T(1.0 / (P.h * P.h)), T(P.omega * P.omega), mv);
                have_st = true;
            }
            const cplx<T>* v = buf + I.sender_buf_off + (int64_t)c * rstride;
            // (beta v)(g + o e_a): zero outside the receiver or the sender window
            auto bv = [&](int ax, int o) -> cplx<T> {
                int gg[3] = {g[0], g[1], g[2]};
                if (ax >= 0) {
                    gg[ax] += o;
                    int xl = gg[ax] - S.lo[ax];
                    if (xl < 0 || xl >= S.nw[ax]) return mk<T>(0, 0);
                }
                T beta = T(1);
                int64_t li = 0;
                for (int a = ndim - 1; a >= 0; --a) {
                    int xl = gg[a] - R.lo[a];
                    if (xl < 0 || xl >= R.nw[a]) return mk<T>(0, 0);
                    li = li * R.nw[a] + xl;
                    beta *= beta1<T>(I.dir[a], gg[a], R.box_lo[a], R.box_hi[a], P.d, tab);
                }
                if (beta == T(0)) return mk<T>(0, 0);
                return beta * v[li];
            };
            cplx<T> Abv = st.diag * bv(-1, 0);
            for (int a = 0; a < ndim; ++a) {
                Abv = Abv + st.cp[a] * bv(a, 1);
                Abv = Abv + st.cm[a] * bv(a, -1);
            }
            val = val - Abv;
        }
    }
    buf[tk.buf_off + (int64_t)c * rstride + k] = val;
}

template <typename T>
void launch_gather(const Task* tasks, int ntask, int64_t max_win, const SubDesc* subs,
                   const Incoming* inc, const DevProblem& P, const T* m, const cplx<T>* an,
                   const cplx<T>* af, const T* beta_tab, const cplx<double>* b, int nrhs,
                   cplx<T>* buf, int64_t rstride, cudaStream_t st) {
    if (ntask == 0) return;
    const int nt = 256;
    dim3 grid((unsigned)((max_win + nt - 1) / nt), ntask, nrhs);
    gather_kernel<T><<<grid, nt, 0, st>>>(tasks, subs, inc, P, m, an, af, beta_tab, b, nrhs,
                                           buf, rstride);
}

// ----------------------------------------------------------------------------- assembly
template <typename T>
__global__ void assemble_kernel(DevProblem P, const SubDesc* __restrict__ subs,
                                const int* __restrict__ box_of, const int64_t* __restrict__ node_buf,
                                int nsweeps, const T* __restrict__ tab,
                                const cplx<T>* __restrict__ buf, int64_t rstride,
                                cplx<double>* U) {
    const int64_t Ng = (int64_t)P.N[0] * P.N[1] * P.N[2];
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (k >= Ng) return;
    const int ndim = P.ndim;
    int g[3];
    g[0] = (int)(k % P.N[0]);
    g[1] = (int)((k / P.N[0]) % P.N[1]);
    g[2] = (int)(k / ((int64_t)P.N[0] * P.N[1]));
    // candidate boxes per axis: own box (cutoff 1) and the neighbour whose
    // cutoff reaches this node
    int cb[3][2];
    T cw[3][2];
    int cn[3];
    int off = 0;
    for (int a = 0; a < 3; ++a) {
        cn[a] = 1;
        cb[a][0] = 0;
        cw[a][0] = T(1);
        if (a >= ndim) continue;
        const int i0 = box_of[off + g[a]];
        off += P.N[a];
        cb[a][0] = i0;
        // neighbour above: its lower cutoff at the m-th node below its face
        if (i0 + 1 < P.nb[a]) {
            int lo1 = -1;
            // find box lo of i0+1 via a subdomain that has it
            int s = 0, stride = 1;
            for (int b2 = 0; b2 < a; ++b2) stride *= P.nb[b2];
            s = (i0 + 1) * stride;
            lo1 = subs[s].box_lo[a];
            int mm = lo1 - 1 - g[a];
            if (mm < P.d) {
                cb[a][cn[a]] = i0 + 1;
                cw[a][cn[a]] = tab[mm];
                ++cn[a];
            }
        }
        if (i0 > 0) {
            int stride = 1;
            for (int b2 = 0; b2 < a; ++b2) stride *= P.nb[b2];
            int hi0 = subs[(i0 - 1) * stride].box_hi[a];
            int mm = g[a] - hi0;
            if (mm < P.d) {
                cb[a][cn[a]] = i0 - 1;
                cw[a][cn[a]] = tab[mm];
                ++cn[a];
            }
        }
    }
    double sr = 0, si = 0;
    for (int i0 = 0; i0 < cn[0]; ++i0)
        for (int i1 = 0; i1 < cn[1]; ++i1)
            for (int i2 = 0; i2 < cn[2]; ++i2) {
                int s = cb[0][i0] + P.nb[0] * (cb[1][i1] + P.nb[1] * cb[2][i2]);
                T wgt = cw[0][i0] * cw[1][i1] * cw[2][i2];
                if (wgt == T(0)) continue;
                const SubDesc& S = subs[s];
                int64_t li = 0;
                for (int a = ndim - 1; a >= 0; --a) li = li * S.nw[a] + (g[a] - S.lo[a]);
                for (int l = 0; l < nsweeps; ++l) {
                    int64_t ob = node_buf[(int64_t)l * P.nsub + s];
                    if (ob < 0) continue;
                    cplx<T> v = buf[ob + (int64_t)c * rstride + li];
                    sr += (double)(wgt * v.re);
                    si += (double)(wgt * v.im);
                }
            }
    U[(int64_t)c * Ng + k] = mk<double>(sr, si);
}

template <typename T>
void launch_assemble(const DevProblem& P, const SubDesc* subs, const int* box_of,
                     const int64_t* node_buf, int nsweeps, const T* beta_tab,
                     const cplx<T>* buf, int64_t rstride, int nrhs, cplx<double>* U,
                     cudaStream_t st) {
    const int64_t Ng = (int64_t)P.N[0] * P.N[1] * P.N[2];
    const int nt = 256;
    dim3 grid((unsigned)((Ng + nt - 1) / nt), nrhs);
    assemble_kernel<T><<<grid, nt, 0, st>>>(P, subs, box_of, node_buf, nsweeps, beta_tab, buf,
                                             rstride, U);
}

template void launch_gather<float>(const Task*, int, int64_t, const SubDesc*, const Incoming*,
                                   const DevProblem&, const float*, const cplx<float>*,
                                   const cplx<float>*, const float*, const cplx<double>*, int,
                                   cplx<float>*, int64_t, cudaStream_t);
template void launch_gather<double>(const Task*, int, int64_t, const SubDesc*, const Incoming*,
                                    const DevProblem&, const double*, const cplx<double>*,
                                    const cplx<double>*, const double*, const cplx<double>*, int,
                                    cplx<double>*, int64_t, cudaStream_t);
template void launch_assemble<float>(const DevProblem&, const SubDesc*, const int*,
                                     const int64_t*, int, const float*, const cplx<float>*,
                                     int64_t, int, cplx<double>*, cudaStream_t);
template void launch_assemble<double>(const DevProblem&, const SubDesc*, const int*,
                                      const int64_t*, int, const double*, const cplx<double>*,
                                      int64_t, int, cplx<double>*, cudaStream_t);

}  // namespace helm
