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
// The elimination is blocked by panels of b columns.  Each Gauss-Jordan step
// k multiplies the array from the left by a row interchange and by a matrix
// that differs from the identity only in column k; moving the interchanges to
// the right, the b steps of a panel K combine into  G P  with G - I nonzero
// only in the columns K.  The panel's own columns are eliminated in shared
// memory (all rows, b columns), after which they hold G[:, K]; every other
// column q then takes the panel's row interchanges and one rank-b update
//     D[:, q] += (G - I)[:, K] D[K, q],
// the complex GEMM that carries all but O(n^2 b) of the O(n^3) work, tiled in
// 4 x 4 register blocks against the panel and the pivot rows in shared memory.
// Each array entry is read and written once per panel instead of once per
// pivot.
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
    cplx<T>* W;      // panel columns [bp][n]
    cplx<T>* V;      // pivot rows [bp][n]
};

// Shared-memory bytes of the factor kernel for blocks of up to nbp rows and
// panels of bp columns (nt threads); the layout follows factor_kernel.
template <typename T>
static size_t factor_smem(int nbp, int ndim, int nt, int bp) {
    const int noff = 2 * (ndim - 1);
    return sizeof(cplx<T>) * (size_t)(6 + noff) * nbp + sizeof(int) * (size_t)(nbp + 2) +
           (sizeof(T) + sizeof(int)) * (size_t)nt + 16 + 2 * sizeof(cplx<T>) * (size_t)bp * nbp + 64;
}

template <typename T>
__device__ __forceinline__ void put(T* D, int nbp, int p, int q, cplx<T> v) {
    D[(int64_t)q * 2 * nbp + p] = v.re;
    D[(int64_t)q * 2 * nbp + nbp + p] = v.im;
}
template <typename T>
__device__ __forceinline__ cplx<T> get(const T* D, int nbp, int p, int q) {
    return mk<T>(D[(int64_t)q * 2 * nbp + p], D[(int64_t)q * 2 * nbp + nbp + p]);
}

// Four consecutive values of one column plane (16-byte aligned: the row offset
// is a multiple of 4 and every plane starts at a multiple of 64 bytes).
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double (&v)[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

// Index of the largest |v|^2 over the CTA (ties: the smaller index); every
// thread passes its candidate and gets the winner.  red: 2 x (nt / 32) words.
template <typename T>
struct ArgMax {
    T v;
    int i;
};
template <typename T>
__device__ __forceinline__ ArgMax<T> block_argmax(T best, int bi, T* rv, int* ri, int tid, int nt) {
    for (int o = 16; o > 0; o >>= 1) {
        const T ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) best = ob, bi = oi;
    }
    if ((tid & 31) == 0) rv[tid >> 5] = best, ri[tid >> 5] = bi;
    __syncthreads();
    if (tid < 32) {
        const int nw = nt >> 5;
        best = tid < nw ? rv[tid] : T(-1);
        bi = tid < nw ? ri[tid] : 0x7fffffff;
        for (int o = 16; o > 0; o >>= 1) {
            const T ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) best = ob, bi = oi;
        }
        if (tid == 0) rv[0] = best, ri[0] = bi;
    }
    __syncthreads();
    const ArgMax<T> r{rv[0], ri[0]};
    __syncthreads();  // rv / ri are reused by the next call
    return r;
}

// In-place inverse of the n x n block D (split planes, leading dimension nbp)
// by Gauss-Jordan elimination with partial row pivoting, blocked by panels of
// bp columns.  W, V: bp x n complex each in shared memory (the panel columns,
// the pivot rows); rowk: bp, colk: n, piv: n, rv / ri: reduction scratch.
template <typename T>
__device__ void gj_invert_blocked(T* D, int nbp, int n, int bp, cplx<T>* W, cplx<T>* V, cplx<T>* rowk,
                                  cplx<T>* colk, int* piv, T* rv, int* ri, int* err) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int k0 = 0; k0 < n; k0 += bp) {
        const int bw = min(bp, n - k0);
        // ---- the panel's columns into shared memory
        for (int e = tid; e < bw * n; e += nt) {
            const int t = e / n, i = e % n;
            W[t * n + i] = get(D, nbp, i, k0 + t);
        }
        __syncthreads();
        // ---- its bw elimination steps on the panel only (every row)
        for (int t = 0; t < bw; ++t) {
            const int k = k0 + t;
            T best = T(-1);
            int bi = k;
            for (int i = k + tid; i < n; i += nt) {
                const T a2 = cabs2(W[t * n + i]);
                if (a2 > best) best = a2, bi = i;
            }
            const ArgMax<T> am = block_argmax(best, bi, rv, ri, tid, nt);
            const T pmag = am.v;
            const int pr = am.i;
            if (tid == 0) piv[k] = pr;
            if (pr != k)
                for (int u = tid; u < bw; u += nt) {
                    const cplx<T> a = W[u * n + k];
                    W[u * n + k] = W[u * n + pr];
                    W[u * n + pr] = a;
                }
            __syncthreads();
            const bool bad = !(pmag > T(0)) || !isfinite(pmag);
            if (bad && tid == 0) atomicExch(err, 1);
            const cplx<T> inv = bad ? mk<T>(0, 0) : cinv(W[t * n + k]);
            for (int u = tid; u < bw; u += nt) rowk[u] = (u == t) ? inv : W[u * n + k] * inv;
            for (int i = tid; i < n; i += nt) colk[i] = (i == k) ? mk<T>(0, 0) : W[t * n + i];
            __syncthreads();
            for (int e = tid; e < bw * n; e += nt) {
                const int u = e / n, i = e % n;
                if (i == k)
                    W[u * n + i] = rowk[u];
                else if (u == t)
                    W[u * n + i] = cneg(colk[i] * inv);
                else
                    W[u * n + i] = W[u * n + i] - colk[i] * rowk[u];
            }
            __syncthreads();
        }
        // ---- the other columns: the panel's interchanges (in order, one column per
        // thread), then the pivot rows into shared memory
        for (int q = tid; q < n; q += nt) {
            if (q >= k0 && q < k0 + bw) continue;
            for (int t = 0; t < bw; ++t) {
                const int k = k0 + t, pr = piv[k];
                if (pr != k) {
                    const cplx<T> a = get(D, nbp, k, q), b = get(D, nbp, pr, q);
                    put(D, nbp, k, q, b);
                    put(D, nbp, pr, q, a);
                }
            }
        }
        __syncthreads();
        for (int e = tid; e < bw * n; e += nt) {
            const int t = e / n, q = e % n;
            V[t * n + q] = (q >= k0 && q < k0 + bw) ? mk<T>(0, 0) : get(D, nbp, k0 + t, q);
        }
        __syncthreads();
        // ---- rank-bw update of the other columns in 4 x 4 blocks:
        //   D[i, q] = (i in K ? 0 : D[i, q]) + sum_t W[t][i] V[t][q]
        const int nrg = (n + 3) / 4, ncg = (n + 3) / 4;
        for (int task = tid; task < nrg * ncg; task += nt) {
            const int i0 = 4 * (task % nrg), q0 = 4 * (task / nrg);
            if (q0 >= k0 && q0 + 3 < k0 + bw) continue;  // all four columns in the panel
            cplx<T> acc[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = mk<T>(0, 0);
            for (int t = 0; t < bw; ++t) {
                cplx<T> w[4], v[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) w[r] = (i0 + r < n) ? W[t * n + i0 + r] : mk<T>(0, 0);
#pragma unroll
                for (int c = 0; c < 4; ++c) v[c] = (q0 + c < n) ? V[t * n + q0 + c] : mk<T>(0, 0);
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        acc[r][c].re += w[r].re * v[c].re - w[r].im * v[c].im;
                        acc[r][c].im += w[r].re * v[c].im + w[r].im * v[c].re;
                    }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int q = q0 + c;
                if (q >= n || (q >= k0 && q < k0 + bw)) continue;
                T* re = D + (int64_t)q * 2 * nbp + i0;
                T* im = re + nbp;
                T vr[4], vi[4];
                ld4(re, vr);
                ld4(im, vi);
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int i = i0 + r;
                    const bool in_k = i >= k0 && i < k0 + bw;
                    if (i < n) {
                        vr[r] = (in_k ? T(0) : vr[r]) + acc[r][c].re;
                        vi[r] = (in_k ? T(0) : vi[r]) + acc[r][c].im;
                    }
                }
                st4(re, vr);
                st4(im, vi);
            }
        }
        // ---- the panel back: its columns now hold G[:, K]
        for (int e = tid; e < bw * n; e += nt) {
            const int t = e / n, i = e % n;
            put(D, nbp, i, k0 + t, W[t * n + i]);
        }
        __syncthreads();
    }
    // ---- undo the row interchanges as column interchanges, last first
    for (int k = n - 1; k >= 0; --k) {
        const int pr = piv[k];
        if (pr != k)
            for (int i = tid; i < n; i += nt) {
                const cplx<T> a = get(D, nbp, i, k), b = get(D, nbp, i, pr);
                put(D, nbp, i, k, b);
                put(D, nbp, i, pr, a);
            }
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(512) factor_kernel(const SubDesc* __restrict__ subs,
                                                     DevProblem P, const T* __restrict__ m,
                                                     const cplx<T>* __restrict__ an,
                                                     const cplx<T>* __restrict__ af, T* fac,
                                                     T* fac2, int twist, int bp, int* err) {
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
    sm.W = reinterpret_cast<cplx<T>*>((reinterpret_cast<uintptr_t>(sm.ri + nt) + 15) & ~uintptr_t(15));
    sm.V = sm.W + (size_t)bp * n;

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
        // ---- Gauss-Jordan inversion in place with partial pivoting, blocked
        gj_invert_blocked(D, nbp, n, bp, sm.W, sm.V, sm.rowk, sm.colk, sm.piv, sm.rv, sm.ri, err);
        for (int p = tid; p < n; p += nt) sm.cprev[p] = sm.ccur[p];
        __syncthreads();
    }
}

// Panel width: the widest of 32, 16, 8, 4, 2, 1 whose panel and pivot rows fit
// in shared memory beside the per-line vectors.
template <typename T>
static int factor_panel(int nbp, int ndim, int nt, size_t* smem) {
    for (int bp = 32; bp >= 1; bp /= 2) {
        *smem = factor_smem<T>(nbp, ndim, nt, bp);
        if (*smem <= 227 * 1024) return bp;
    }
    return 1;
}

template <typename T>
static void launch_factor_t(const SubDesc* subs, int nsub, int nbp_max, const DevProblem& P,
                            const T* m, const cplx<T>* an, const cplx<T>* af, T* fac, T* fac2, int twist,
                            int* err, cudaStream_t st) {
    const int nt = 512;
    size_t smem = 0;
    const int bp = factor_panel<T>(nbp_max, P.ndim, nt, &smem);
    cudaFuncSetAttribute(factor_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    factor_kernel<T><<<nsub, nt, smem, st>>>(subs, P, m, an, af, fac, fac2, twist, bp, err);
}

void launch_factor_twist_f32(const SubDesc* subs, int nsub, int nbp_max, const DevProblem& P,
                             const float* m32, const cplx<float>* an, const cplx<float>* af,
                             const float* fac, float* fac2, int* err, cudaStream_t st) {
    launch_factor_t<float>(subs, nsub, nbp_max, P, m32, an, af, const_cast<float*>(fac), fac2, 1, err, st);
}

void launch_factor_f32(const SubDesc* subs, int nsub, int nbp_max, const DevProblem& P,
                       const float* m32, const cplx<float>* an, const cplx<float>* af,
                       float* fac, int* err, cudaStream_t st) {
    launch_factor_t<float>(subs, nsub, nbp_max, P, m32, an, af, fac, nullptr, 0, err, st);
}
void launch_factor_f64(const SubDesc* subs, int nsub, int nbp_max, const DevProblem& P,
                       const double* m64, const cplx<double>* an, const cplx<double>* af,
                       double* fac, int* err, cudaStream_t st) {
    launch_factor_t<double>(subs, nsub, nbp_max, P, m64, an, af, fac, nullptr, 0, err, st);
}

}  // namespace helm
