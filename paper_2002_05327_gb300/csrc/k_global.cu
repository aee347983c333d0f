// Global FP64 kernels: J scaling of sources, the residual b - A u of the
// global PML system (Eq. 2.2, J-multiplied 5/7-point form), the batched
// BLAS-1 of GMRES (one Krylov space per right-hand side) and the gradient of
// the receiver misfit with respect to m.
//
// Reductions are deterministic: every block reduces a fixed contiguous chunk
// with a fixed tree, and a second pass sums the block partials in order.
//
// The operator product and the Gram-Schmidt kernels (multi-vector dots,
// combinations, norms) keep their vectors in FP64 but do their arithmetic in
// float-float ("double-float" pairs hi + lo) on the FP32 pipes: on this GPU
// the FP64 pipe issues about one sixty-fourth of the FP32 rate, and the FP64
// versions of these kernels ran at ~87% of it.  A double is split exactly
// into its top 24 and next 24 mantissa bits, and a result recombined, with
// integer operations only (ff.h: conversions and additions in FP64 would use
// the FP64 pipe); products are formed exactly with FMA (TwoProd) and sums are
// compensated (TwoSum), so a dot or combination carries ~48 significant bits
// -- ample for an Arnoldi relation to the 1e-8 residual the solver targets.
#include "helm_internal.h"
#include "ff.h"

namespace helm {

using namespace ffa;

__device__ __forceinline__ void unflat(int64_t k, const int N[3], int g[3]) {
    g[0] = (int)(k % N[0]);
    g[1] = (int)((k / N[0]) % N[1]);
    g[2] = (int)(k / ((int64_t)N[0] * N[1]));
}

__global__ void scale_J_kernel(DevProblem P, Win<double> w, const cplx<double>* f,
                               cplx<double>* b, int nrhs, int conj_in) {
    const int64_t Ng = (int64_t)P.N[0] * P.N[1] * P.N[2];
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (k >= Ng) return;
    int g[3];
    unflat(k, P.N, g);
    cplx<double> J = mk<double>(1, 0);
    for (int a = 0; a < P.ndim; ++a) J = J * w.alpha_node[a][g[a]];
    cplx<double> v = f[(int64_t)c * Ng + k];
    if (conj_in) v = cconj(v);
    b[(int64_t)c * Ng + k] = J * v;
}

void launch_scale_J(const DevProblem& P, const Win<double>& g, const cplx<double>* f,
                    cplx<double>* b, int nrhs, bool conj_in, cudaStream_t st) {
    const int64_t Ng = (int64_t)P.N[0] * P.N[1] * P.N[2];
    dim3 grid((unsigned)((Ng + 255) / 256), nrhs);
    scale_J_kernel<<<grid, 256, 0, st>>>(P, g, f, b, nrhs, conj_in ? 1 : 0);
}

// The J-multiplied stencil of every grid node (diagonal, then the +/- neighbour
// of each axis), formed once in FP64 and stored as float-float pairs
// (re.hi, re.lo, im.hi, im.lo): the operator product then needs no FP64
// instruction.
__global__ void stencil_ff_kernel(DevProblem P, Win<double> w, const double* __restrict__ m, double ih2,
                                  double om2, float4* __restrict__ stc) {
    const int64_t Ng = (int64_t)P.N[0] * P.N[1] * P.N[2];
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Ng) return;
    int g[3];
    unflat(k, P.N, g);
    const Stencil<double> st = stencil_at(w, P.ndim, g, ih2, om2, m[k]);
    const int npt = 1 + 2 * P.ndim;
    auto put = [&](int i, cplx<double> v) {
        const ff r = split_d(v.re), im = split_d(v.im);
        stc[k * npt + i] = make_float4(r.hi, r.lo, im.hi, im.lo);
    };
    put(0, st.diag);
    for (int a = 0; a < P.ndim; ++a) {
        put(1 + 2 * a, st.cp[a]);
        put(2 + 2 * a, st.cm[a]);
    }
}

void launch_stencil_ff(const DevProblem& P, const Win<double>& g, const double* m, float4* stc,
                       cudaStream_t st) {
    const int64_t Ng = (int64_t)P.N[0] * P.N[1] * P.N[2];
    stencil_ff_kernel<<<(unsigned)((Ng + 255) / 256), 256, 0, st>>>(P, g, m, 1.0 / (P.h * P.h),
                                                                     P.omega * P.omega, stc);
}

// b - A u (or -A u without b), one thread per grid node: the node's stencil
// (float-float, from stencil_ff_kernel) is read once and applied to every
// right-hand side in float-float arithmetic on the FP32 pipes (vectors stay
// FP64 in memory).  Outside the PML every alpha is 1, so the coefficients are
// real (their imaginary parts are exact zeros) and each term needs two
// products, not four.
__global__ void apply_A_kernel(DevProblem P, const float4* __restrict__ stc, const cplx<double>* __restrict__ b,
                               const cplx<double>* __restrict__ u, cplx<double>* __restrict__ r, int nrhs) {
    const int64_t Ng = (int64_t)P.N[0] * P.N[1] * P.N[2];
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Ng) return;
    int g[3];
    unflat(k, P.N, g);
    const int npt = 1 + 2 * P.ndim;
    const float4* sk = stc + k * npt;
    int64_t off[6];
    ff cr[6], ci[6];
    int np = 0;
    int64_t stride = 1;
    for (int a = 0; a < P.ndim; ++a) {
        if (g[a] + 1 < P.N[a]) {
            const float4 q = sk[1 + 2 * a];
            off[np] = stride;
            cr[np] = {q.x, q.y};
            ci[np++] = {q.z, q.w};
        }
        if (g[a] > 0) {
            const float4 q = sk[2 + 2 * a];
            off[np] = -stride;
            cr[np] = {q.x, q.y};
            ci[np++] = {q.z, q.w};
        }
        stride *= P.N[a];
    }
    const float4 q0 = sk[0];
    const ff dr = {q0.x, q0.y}, di = {q0.z, q0.w};
    bool real = di.hi == 0.f;
    for (int i = 0; i < np; ++i) real = real && ci[i].hi == 0.f;
    for (int c = 0; c < nrhs; ++c) {
        const cplx<double>* uc = u + (int64_t)c * Ng + k;
        // -(A u) accumulated, then + b
        ff ar = {0.f, 0.f}, ai = {0.f, 0.f};
        if (b) {
            const cplx<double> bv = b[(int64_t)c * Ng + k];
            ar = split_d(bv.re);
            ai = split_d(bv.im);
        }
        const cplx<double> u0 = uc[0];
        const ff ur = split_d(u0.re), ui = split_d(u0.im);
        acc_mul(ar, ff_neg(dr), ur);
        acc_mul(ai, ff_neg(dr), ui);
        if (!real) {
            acc_mul(ar, di, ui);
            acc_mul(ai, ff_neg(di), ur);
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            if (i >= np) break;
            const cplx<double> un = uc[off[i]];
            const ff nr = split_d(un.re), ni = split_d(un.im);
            acc_mul(ar, ff_neg(cr[i]), nr);
            acc_mul(ai, ff_neg(cr[i]), ni);
            if (!real) {
                acc_mul(ar, ci[i], ni);
                acc_mul(ai, ff_neg(ci[i]), nr);
            }
        }
        r[(int64_t)c * Ng + k] = mk<double>(join_d(ar), join_d(ai));
    }
}

void launch_apply_A(const DevProblem& P, const float4* stc, const cplx<double>* b, const cplx<double>* u,
                    cplx<double>* r, int nrhs, cudaStream_t st) {
    const int64_t Ng = (int64_t)P.N[0] * P.N[1] * P.N[2];
    apply_A_kernel<<<(unsigned)((Ng + 255) / 256), 256, 0, st>>>(P, stc, b, u, r, nrhs);
}

// ---- batched dots: out[i*nrhs + c] = sum_k conj(V_i[c][k]) w[c][k]
constexpr int DOT_NT = 256;

__global__ void dots_partial_kernel(const cplx<double>* __restrict__ V, int64_t vstride,
                                    const cplx<double>* __restrict__ w, int64_t n, int nrhs,
                                    cplx<double>* partial, int nblk) {
    __shared__ double sr[DOT_NT], si[DOT_NT];
    const int blk = blockIdx.x;
    const int i = blockIdx.y / nrhs, c = blockIdx.y % nrhs;
    const int64_t chunk = (n + nblk - 1) / nblk;
    const int64_t k0 = (int64_t)blk * chunk;
    const int64_t k1 = min(n, k0 + chunk);
    const cplx<double>* vi = V + (int64_t)i * vstride + (int64_t)c * n;
    const cplx<double>* wc = w + (int64_t)c * n;
    double ar = 0, ai = 0;
    for (int64_t k = k0 + threadIdx.x; k < k1; k += DOT_NT) {
        cplx<double> a = vi[k], b = wc[k];
        ar += a.re * b.re + a.im * b.im;
        ai += a.re * b.im - a.im * b.re;
    }
    sr[threadIdx.x] = ar;
    si[threadIdx.x] = ai;
    __syncthreads();
    for (int s = DOT_NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sr[threadIdx.x] += sr[threadIdx.x + s];
            si[threadIdx.x] += si[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[(int64_t)blockIdx.y * nblk + blk] = mk<double>(sr[0], si[0]);
}

__global__ void dots_final_kernel(const cplx<double>* partial, int nblk, int count,
                                  cplx<double>* out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    double r = 0, i = 0;
    for (int b = 0; b < nblk; ++b) {
        r += partial[(int64_t)t * nblk + b].re;
        i += partial[(int64_t)t * nblk + b].im;
    }
    out[t] = mk<double>(r, i);
}

void launch_dots(const cplx<double>* V, int64_t vstride, int nv, const cplx<double>* w,
                 int64_t n, int nrhs, cplx<double>* out, cplx<double>* partial, int nblk,
                 cudaStream_t st) {
    dim3 grid(nblk, nv * nrhs);
    dots_partial_kernel<<<grid, DOT_NT, 0, st>>>(V, vstride, w, n, nrhs, partial, nblk);
    int count = nv * nrhs;
    dots_final_kernel<<<(count + 127) / 128, 128, 0, st>>>(partial, nblk, count, out);
}

// w[c] += sign * sum_i coef[i*nrhs+c] V_i[c]
__global__ void sub_combo_kernel(cplx<double>* w, const cplx<double>* __restrict__ V,
                                 int64_t vstride, int nv, const cplx<double>* __restrict__ coef,
                                 int64_t n, int nrhs, double sign) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (k >= n) return;
    cplx<double> acc = w[(int64_t)c * n + k];
    for (int i = 0; i < nv; ++i) {
        cplx<double> a = coef[i * nrhs + c];
        cplx<double> v = V[(int64_t)i * vstride + (int64_t)c * n + k];
        acc = acc + sign * (a * v);
    }
    w[(int64_t)c * n + k] = acc;
}

void launch_sub_combo(cplx<double>* w, const cplx<double>* V, int64_t vstride, int nv,
                      const cplx<double>* coef, int64_t n, int nrhs, double sign,
                      cudaStream_t st) {
    dim3 grid((unsigned)((n + 255) / 256), nrhs);
    sub_combo_kernel<<<grid, 256, 0, st>>>(w, V, vstride, nv, coef, n, nrhs, sign);
}

__global__ void scale_vec_kernel(cplx<double>* v, const cplx<double>* src, const double* s,
                                 int64_t n) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (k >= n) return;
    v[(int64_t)c * n + k] = s[c] * src[(int64_t)c * n + k];
}

void launch_scale_vec(cplx<double>* v, const cplx<double>* src, const double* s, int64_t n,
                      int nrhs, cudaStream_t st) {
    dim3 grid((unsigned)((n + 255) / 256), nrhs);
    scale_vec_kernel<<<grid, 256, 0, st>>>(v, src, s, n);
}

__global__ void conj_kernel(cplx<double>* v, int64_t count) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < count) v[k].im = -v[k].im;
}

// ---- fused multi-vector kernels of classical Gram-Schmidt: one pass over w
// and every V_i (V given as a device array of pointers)

__global__ void mdots_partial_kernel(const cplx<double>* const* __restrict__ V, int nv,
                                     const cplx<double>* __restrict__ w, int64_t n, int nrhs,
                                     cplx<double>* partial, int nblk) {
    __shared__ ff sr[8][DOT_NT / 32], si[8][DOT_NT / 32];
    const int blk = blockIdx.x, c = blockIdx.y, i0 = blockIdx.z * 8;
    const int nvb = min(8, nv - i0);
    const int64_t chunk = (n + nblk - 1) / nblk;
    const int64_t k0 = (int64_t)blk * chunk, k1 = min(n, k0 + chunk);
    const cplx<double>* wc = w + (int64_t)c * n;
    ff ar[8], ai[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) ar[i] = ai[i] = ff{0.f, 0.f};
    for (int64_t k = k0 + threadIdx.x; k < k1; k += DOT_NT) {
        const cplx<double> bw = wc[k];
        const ff br = split_d(bw.re), bi = split_d(bw.im);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (i < nvb) {
                const cplx<double> av = V[i0 + i][(int64_t)c * n + k];
                const ff vr = split_d(av.re), vi = split_d(av.im);
                // conj(v) w = (vr br + vi bi) + i (vr bi - vi br)
                acc_mul(ar[i], vr, br);
                acc_mul(ar[i], vi, bi);
                acc_mul(ai[i], vr, bi);
                acc_mul(ai[i], ff_neg(vi), br);
            }
        }
    }
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        for (int o = 16; o > 0; o >>= 1) {
            ar[i] = ff_sum(ar[i], shfl_down_ff(ar[i], o));
            ai[i] = ff_sum(ai[i], shfl_down_ff(ai[i], o));
        }
        if (lane == 0) {
            sr[i][wp] = ar[i];
            si[i][wp] = ai[i];
        }
    }
    __syncthreads();
    if (threadIdx.x < nvb) {
        const int i = threadIdx.x;
        ff r = {0.f, 0.f}, im = {0.f, 0.f};
        for (int q = 0; q < DOT_NT / 32; ++q) {
            r = ff_sum(r, sr[i][q]);
            im = ff_sum(im, si[i][q]);
        }
        partial[((int64_t)(i0 + i) * nrhs + c) * nblk + blk] = mk<double>(join_d(r), join_d(im));
    }
}

// squared norms |v[c]|^2 into out[c] (imaginary part 0), float-float
__global__ void norms_partial_kernel(const cplx<double>* __restrict__ v, int64_t n,
                                     cplx<double>* partial, int nblk) {
    __shared__ ff sr[DOT_NT / 32];
    const int blk = blockIdx.x, c = blockIdx.y;
    const int64_t chunk = (n + nblk - 1) / nblk;
    const int64_t k0 = (int64_t)blk * chunk, k1 = min(n, k0 + chunk);
    const cplx<double>* vc = v + (int64_t)c * n;
    ff a = {0.f, 0.f};
    for (int64_t k = k0 + threadIdx.x; k < k1; k += DOT_NT) {
        const cplx<double> x = vc[k];
        const ff xr = split_d(x.re), xi = split_d(x.im);
        acc_mul(a, xr, xr);
        acc_mul(a, xi, xi);
    }
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) a = ff_sum(a, shfl_down_ff(a, o));
    if (lane == 0) sr[wp] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        ff r = {0.f, 0.f};
        for (int q = 0; q < DOT_NT / 32; ++q) r = ff_sum(r, sr[q]);
        partial[(int64_t)c * nblk + blk] = mk<double>(join_d(r), 0.0);
    }
}

void launch_norms2(const cplx<double>* v, int64_t n, int nrhs, cplx<double>* out,
                   cplx<double>* partial, int nblk, cudaStream_t st) {
    dim3 grid(nblk, nrhs);
    norms_partial_kernel<<<grid, DOT_NT, 0, st>>>(v, n, partial, nblk);
    dots_final_kernel<<<(nrhs + 127) / 128, 128, 0, st>>>(partial, nblk, nrhs, out);
}

void launch_mdots(const cplx<double>* const* V, int nv, const cplx<double>* w, int64_t n, int nrhs,
                  cplx<double>* out, cplx<double>* partial, int nblk, cudaStream_t st) {
    dim3 grid(nblk, nrhs, (nv + 7) / 8);
    mdots_partial_kernel<<<grid, DOT_NT, 0, st>>>(V, nv, w, n, nrhs, partial, nblk);
    int count = nv * nrhs;
    dots_final_kernel<<<(count + 127) / 128, 128, 0, st>>>(partial, nblk, count, out);
}

// w[c] += sign * sum_i coef[i*nrhs+c] V_i[c], accumulated in float-float; the
// block's coefficients (one right-hand side per block row) are split once into
// shared memory
__global__ void mcombo_kernel(cplx<double>* w, const cplx<double>* const* __restrict__ V, int nv,
                              const cplx<double>* __restrict__ coef, int64_t n, int nrhs,
                              double sign) {
    __shared__ ff scr[64], sci[64];
    const int c = blockIdx.y;
    const float sg = sign < 0 ? -1.f : 1.f;  // sign is +-1
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
        const cplx<double> a = coef[i * nrhs + c];
        const ff cr = split_d(a.re), ci = split_d(a.im);
        scr[i] = {sg * cr.hi, sg * cr.lo};
        sci[i] = {sg * ci.hi, sg * ci.lo};
    }
    __syncthreads();
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const cplx<double> w0 = w[(int64_t)c * n + k];
    ff ar = split_d(w0.re), ai = split_d(w0.im);
    for (int i = 0; i < nv; ++i) {
        const ff cr = scr[i], ci = sci[i];
        const cplx<double> v = V[i][(int64_t)c * n + k];
        const ff vr = split_d(v.re), vi = split_d(v.im);
        // (cr + i ci)(vr + i vi)
        acc_mul(ar, cr, vr);
        acc_mul(ar, ff_neg(ci), vi);
        acc_mul(ai, cr, vi);
        acc_mul(ai, ci, vr);
    }
    w[(int64_t)c * n + k] = mk<double>(join_d(ar), join_d(ai));
}

void launch_mcombo(cplx<double>* w, const cplx<double>* const* V, int nv, const cplx<double>* coef,
                   int64_t n, int nrhs, double sign, cudaStream_t st) {
    dim3 grid((unsigned)((n + 255) / 256), nrhs);
    mcombo_kernel<<<grid, 256, 0, st>>>(w, V, nv, coef, n, nrhs, sign);
}

void launch_conj(cplx<double>* v, int64_t count, cudaStream_t st) {
    conj_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(v, count);
}

__global__ void gradient_kernel(DevProblem P, Win<double> w, const cplx<double>* __restrict__ U,
                                const cplx<double>* __restrict__ L, int nsrc, double* grad) {
    const int64_t Ng = (int64_t)P.N[0] * P.N[1] * P.N[2];
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Ng) return;
    int g[3];
    unflat(k, P.N, g);
    cplx<double> J = mk<double>(1, 0);
    for (int a = 0; a < P.ndim; ++a) J = J * w.alpha_node[a][g[a]];
    double acc = 0;
    for (int s = 0; s < nsrc; ++s) {
        cplx<double> t = cconj(L[(int64_t)s * Ng + k]) * (J * U[(int64_t)s * Ng + k]);
        acc += t.re;
    }
    grad[k] = -P.omega * P.omega * acc;
}

void launch_gradient(const DevProblem& P, const Win<double>& g, const cplx<double>* U,
                     const cplx<double>* L, int nsrc, double* grad, cudaStream_t st) {
    const int64_t Ng = (int64_t)P.N[0] * P.N[1] * P.N[2];
    gradient_kernel<<<(unsigned)((Ng + 255) / 256), 256, 0, st>>>(P, g, U, L, nsrc, grad);
}

}  // namespace helm
