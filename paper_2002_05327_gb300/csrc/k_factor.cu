// Block-tridiagonal block LU of every subdomain PML operator (the local
// problems P_{Omega_ij} of Algorithm 3.1 / 4.1).
//
// A subdomain window is ordered block by block along its slowest axis
// (lines in 2D, planes in 3D).  With A_jj the block of line j and the
// diagonal couplings a_j (to line j-1) and c_j (to line j+1):
//     S_0 = A_00,   S_j = A_jj - diag(a_j) D_{j-1} diag(c_{j-1}),   D_j = S_j^{-1}.
// D_j is formed densely and inverted in place by Gauss-Jordan elimination with
// partial (row) pivoting; the row interchanges are undone as column
// interchanges at the end.
//
// Storage of D_j (n x n, padded to nbp): column-major, split planes:
//     re(p,q) = base[q*2*nbp + p],  im(p,q) = base[q*2*nbp + nbp + p]
// so that a warp reading rows p..p+31 of one column is coalesced.
//
// One CTA per subdomain; all subdomains are independent and run in one launch.
// The working matrix lives in the factor storage (L2-resident during its line).
//
// Twisted mode (for the two-ended solve of the tensor-core path): with
// mid = nlines / 2, the lines below mid are eliminated from the far end,
//     T_{nl-1} = A,   T_j = A_jj - diag(c_j) E_{j+1} diag(c_j),   E_j = T_j^{-1}   (j > mid),
// and the middle line takes both Schur complements,
//     M = A_mm - diag(a_m) D_{mid-1} diag(a_m) - diag(c_m) E_{mid+1} diag(c_m),   F = M^{-1},
// where D_{mid-1} comes from the standard factors.  The operator is complex
// symmetric, so the coupling of line j to j+1 equals that of j+1 to j
// (c_j = a_{j+1}, computed from the same face coefficient) and every term uses
// line j's own stencil.  E_j and F are written to a second array of the same
// layout (lines mid .. nl-1).
#include "helm_internal.h"

namespace helm {

template <typename T>
struct FacSmem {
    cplx<T>* rowk;   // pivot row scaled by 1/pivot
    cplx<T>* colk;   // multipliers of the pivot column
    cplx<T>* cprev;  // c_{j-1}
    cplx<T>* acur;   // a_j
    cplx<T>* ccur;   // c_j
    cplx<T>* diag;   // diagonal of A_jj
    cplx<T>* off;    // off-diagonals of A_jj: [2*(ndim-1)][n]
    int* piv;
    T* rv;           // reduction values
    int* ri;         // reduction indices
};

template <typename T>
__device__ __forceinline__ void put(T* D, int nbp, int p, int q, cplx<T> v) {
    D[(int64_t)q * 2 * nbp + p] = v.re;
    D[(int64_t)q * 2 * nbp + nbp + p] = v.im;
}
template <typename T>
__device__ __forceinline__ cplx<T> get(const T* D, int nbp, int p, int q) {
    return mk<T>(D[(int64_t)q * 2 * nbp + p], D[(int64_t)q * 2 * nbp + nbp + p]);
}

template <typename T>
__global__ void __launch_bounds__(512) factor_kernel(const SubDesc* __restrict__ subs,
                                                     DevProblem P, const T* __restrict__ m,
                                                     const cplx<T>* __restrict__ an,
                                                     const cplx<T>* __restrict__ af, T* fac,
                                                     T* fac2, int twist, int* err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SubDesc S = subs[blockIdx.x];
    const int ndim = P.ndim;
    const int n = S.nblk, nbp = S.nbp, slow = ndim - 1;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int noff = 2 * (ndim - 1);

    FacSmem<T> sm;
    cplx<T>* cs = reinterpret_cast<cplx<T>*>(smem_raw);
    sm.rowk = cs;
    sm.colk = cs + n;
    sm.cprev = cs + 2 * n;
    sm.acur = cs + 3 * n;
    sm.ccur = cs + 4 * n;
    sm.diag = cs + 5 * n;
    sm.off = cs + 6 * n;
    sm.piv = reinterpret_cast<int*>(cs + (6 + noff) * n);
    sm.rv = reinterpret_cast<T*>(sm.piv + n + (n & 1));
    sm.ri = reinterpret_cast<int*>(sm.rv + nt);

    Win<T> w;
    for (int a = 0; a < 3; ++a) {
        w.lo[a] = S.lo[a];
        w.n[a] = S.nw[a];
        w.alpha_node[a] = an + S.alpha_off[a];
        w.alpha_face[a] = af + S.face_off[a];
    }
    const T inv_h2 = T(1.0 / (P.h * P.h));
    const T omega2 = T(P.omega * P.omega);
    const int nw0 = S.nw[0];

    const int nl = S.nlines, mid = nl / 2;
    const int nsteps = twist ? nl - mid : nl;
    const int64_t lstride = (int64_t)2 * nbp * nbp;
    for (int t = 0; t < nsteps; ++t) {
        // standard: line t of fac, Schur term from line t-1 of fac;
        // twisted: lines nl-1 .. mid+1 then mid of fac2
        const int j = !twist ? t : (t < nl - 1 - mid ? nl - 1 - t : mid);
        T* D = (twist ? fac2 : fac) + S.fac_off + (int64_t)j * lstride;
        const T* Dp = fac + S.fac_off + (int64_t)(j - 1) * lstride;                         // D_{j-1}
        const T* Ep = (twist ? fac2 : fac) + S.fac_off + (int64_t)(j + 1) * lstride;     // E_{j+1}
        const bool sch_top = !twist ? j > 0 : (j == mid && mid >= 1);
        const bool sch_bot = twist && j + 1 <= nl - 1;
        // ---- stencil rows of line j
        for (int p = tid; p < n; p += nt) {
            int x[3] = {0, 0, 0};
            if (ndim == 2) {
                x[0] = p;
                x[1] = j;
            } else {
                x[0] = p % nw0;
                x[1] = p / nw0;
                x[2] = j;
            }
            int g[3] = {S.lo[0] + x[0], S.lo[1] + x[1], ndim == 3 ? S.lo[2] + x[2] : 0};
            T mv = m[((int64_t)g[2] * P.N[1] + g[1]) * P.N[0] + g[0]];
            Stencil<T> st = stencil_at(w, ndim, x, inv_h2, omega2, mv);
            sm.diag[p] = st.diag;
            sm.acur[p] = st.cm[slow];
            sm.ccur[p] = st.cp[slow];
            for (int a = 0; a < ndim - 1; ++a) {
                sm.off[(2 * a) * n + p] = st.cp[a];
                sm.off[(2 * a + 1) * n + p] = st.cm[a];
            }
        }
        __syncthreads();
        // ---- S_j = A_jj - diag(a_j) D_{j-1} diag(c_{j-1})
        for (int64_t e = tid; e < (int64_t)n * n; e += nt) {
            int q = (int)(e / n), p = (int)(e % n);
            cplx<T> v = mk<T>(0, 0);
            if (p == q) {
                v = sm.diag[p];
            } else {
                int dpq = q - p;
                if (dpq == 1 && (p % nw0) != nw0 - 1) v = sm.off[p];
                if (dpq == -1 && (p % nw0) != 0) v = sm.off[n + p];
                if (ndim == 3) {
                    if (dpq == nw0) v = sm.off[2 * n + p];
                    if (dpq == -nw0) v = sm.off[3 * n + p];
                }
            }
            if (sch_top) v = v - sm.acur[p] * get(Dp, nbp, p, q) * (twist ? sm.acur[q] : sm.cprev[q]);
            if (sch_bot) v = v - sm.ccur[p] * get(Ep, nbp, p, q) * sm.ccur[q];
            put(D, nbp, p, q, v);
        }
        __syncthreads();
        // ---- Gauss-Jordan inversion in place with partial pivoting
        for (int k = 0; k < n; ++k) {
            T best = T(-1);
            int bi = k;
            for (int i = k + tid; i < n; i += nt) {
                cplx<T> v = get(D, nbp, i, k);
                T a2 = cabs2(v);
                if (a2 > best) {
                    best = a2;
                    bi = i;
                }
            }
            sm.rv[tid] = best;
            sm.ri[tid] = bi;
            __syncthreads();
            for (int s = nt / 2; s > 0; s >>= 1) {
                if (tid < s) {
                    T o = sm.rv[tid + s];
                    int oi = sm.ri[tid + s];
                    if (o > sm.rv[tid] || (o == sm.rv[tid] && oi < sm.ri[tid])) {
                        sm.rv[tid] = o;
                        sm.ri[tid] = oi;
                    }
                }
                __syncthreads();
            }
            const int pr = sm.ri[0];
            const T pmag = sm.rv[0];
            if (tid == 0) sm.piv[k] = pr;
            if (pr != k) {
                for (int q = tid; q < n; q += nt) {
                    cplx<T> a = get(D, nbp, k, q), b = get(D, nbp, pr, q);
                    put(D, nbp, k, q, b);
                    put(D, nbp, pr, q, a);
                }
            }
            __syncthreads();
            cplx<T> pv = get(D, nbp, k, k);
            bool bad = !(pmag > T(0)) || !isfinite(pmag);
            if (bad && tid == 0) atomicExch(err, 1);
            cplx<T> inv = bad ? mk<T>(0, 0) : cinv(pv);
            for (int q = tid; q < n; q += nt) {
                sm.rowk[q] = (q == k) ? inv : get(D, nbp, k, q) * inv;
                sm.colk[q] = (q == k) ? mk<T>(0, 0) : get(D, nbp, q, k);
            }
            __syncthreads();
            for (int64_t e = tid; e < (int64_t)n * n; e += nt) {
                int q = (int)(e / n), i = (int)(e % n);
                if (i == k) {
                    put(D, nbp, k, q, sm.rowk[q]);
                } else if (q == k) {
                    put(D, nbp, i, k, cneg(sm.colk[i] * inv));
                } else {
                    cplx<T> f = sm.colk[i];
                    if (f.re != T(0) || f.im != T(0)) put(D, nbp, i, q, get(D, nbp, i, q) - f * sm.rowk[q]);
                }
            }
            __syncthreads();
        }
        // ---- undo the row interchanges as column interchanges, last first
        for (int k = n - 1; k >= 0; --k) {
            int pr = sm.piv[k];
            if (pr != k) {
                for (int i = tid; i < n; i += nt) {
                    cplx<T> a = get(D, nbp, i, k), b = get(D, nbp, i, pr);
                    put(D, nbp, i, k, b);
                    put(D, nbp, i, pr, a);
                }
            }
            __syncthreads();
        }
        for (int p = tid; p < n; p += nt) sm.cprev[p] = sm.ccur[p];
        __syncthreads();
    }
}

template <typename T>
static void launch_factor_t(const SubDesc* subs, int nsub, int nbp_max, const DevProblem& P,
                            const T* m, const cplx<T>* an, const cplx<T>* af, T* fac, int* err,
                            cudaStream_t st) {
    const int nt = 512;
    const int noff = 2 * (P.ndim - 1);
    size_t smem = sizeof(cplx<T>) * (size_t)(6 + noff) * nbp_max + sizeof(int) * (nbp_max + 2) +
                  (sizeof(T) + sizeof(int)) * nt + 64;
    cudaFuncSetAttribute(factor_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    factor_kernel<T><<<nsub, nt, smem, st>>>(subs, P, m, an, af, fac, nullptr, 0, err);
}

void launch_factor_twist_f32(const SubDesc* subs, int nsub, int nbp_max, const DevProblem& P,
                             const float* m32, const cplx<float>* an, const cplx<float>* af,
                             const float* fac, float* fac2, int* err, cudaStream_t st) {
    const int nt = 512;
    const int noff = 2 * (P.ndim - 1);
    size_t smem = sizeof(cplx<float>) * (size_t)(6 + noff) * nbp_max + sizeof(int) * (nbp_max + 2) +
                  (sizeof(float) + sizeof(int)) * nt + 64;
    cudaFuncSetAttribute(factor_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    factor_kernel<float><<<nsub, nt, smem, st>>>(subs, P, m32, an, af, const_cast<float*>(fac), fac2, 1,
                                                 err);
}

void launch_factor_f32(const SubDesc* subs, int nsub, int nbp_max, const DevProblem& P,
                       const float* m32, const cplx<float>* an, const cplx<float>* af,
                       float* fac, int* err, cudaStream_t st) {
    launch_factor_t<float>(subs, nsub, nbp_max, P, m32, an, af, fac, err, st);
}
void launch_factor_f64(const SubDesc* subs, int nsub, int nbp_max, const DevProblem& P,
                       const double* m64, const cplx<double>* an, const cplx<double>* af,
                       double* fac, int* err, cudaStream_t st) {
    launch_factor_t<double>(subs, nsub, nbp_max, P, m64, an, af, fac, err, st);
}

}  // namespace helm
