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

// b = J f (or J conj(f)): one thread per grid node, J = prod_a alpha_a formed
// once and applied to every right-hand side (coalesced along the nodes for
// each right-hand side); the FP64 products of J are not repeated per RHS.
constexpr int kSJ = 8;  // right-hand sides per thread
__global__ void scale_J_kernel(DevProblem P, Win<double> w, const cplx<double>* __restrict__ f,
                               cplx<double>* __restrict__ b, int nrhs, int conj_in) {
    const int64_t Ng = (int64_t)P.N[0] * P.N[1] * P.N[2];
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Ng) return;
    int g[3];
    unflat(k, P.N, g);
    cplx<double> J = mk<double>(1, 0);
    for (int a = 0; a < P.ndim; ++a) J = J * w.alpha_node[a][g[a]];
    const int c1 = min(nrhs, (int)(blockIdx.y + 1) * kSJ);
    for (int c = blockIdx.y * kSJ; c < c1; ++c) {
        cplx<double> v = f[(int64_t)c * Ng + k];
        if (conj_in) v = cconj(v);
        b[(int64_t)c * Ng + k] = J * v;
    }
}

void launch_scale_J(const DevProblem& P, const Win<double>& g, const cplx<double>* f,
                    cplx<double>* b, int nrhs, bool conj_in, cudaStream_t st) {
    const int64_t Ng = (int64_t)P.N[0] * P.N[1] * P.N[2];
    dim3 grid((unsigned)((Ng + 255) / 256), (nrhs + kSJ - 1) / kSJ);
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

// b - A u (or -A u without b).  One thread per (grid node, pair of
// right-hand sides): the node's stencil (float-float, from stencil_ff_kernel)
// is read once and applied to both in float-float arithmetic on the FP32
// pipes, their loads issued together.  The pairs are the fast grid axis, so
// the blocks of one node range run together and share its stencil and
// neighbour rows through L2 (node ranges fastest re-read the stencil from DRAM
// once per pair).  u and r are complex128 (the caller's
// arrays) or float-float (the Krylov work vectors).  Outside the PML every
// alpha is 1, so the coefficients are real (their imaginary parts are exact
// zeros) and each term needs two products, not four.
constexpr int kAR = 2;  // right-hand sides per thread of the operator product
// Grid coordinates of node k of an NDIM-dimensional grid, in 32-bit integer
// arithmetic where the grid has fewer than 2^32 nodes (uniform over a launch);
// a 64-bit division is a long software sequence on the GPU.
template <int NDIM>
__device__ __forceinline__ void unflat_nd(int64_t k, const int N[3], bool small, int g[3]) {
    if (small) {
        const uint32_t kk = (uint32_t)k, n0 = (uint32_t)N[0];
        const uint32_t q = kk / n0;
        g[0] = (int)(kk - q * n0);
        if (NDIM == 2) {
            g[1] = (int)q;
            g[2] = 0;
        } else {
            const uint32_t n1 = (uint32_t)N[1], q2 = q / n1;
            g[1] = (int)(q - q2 * n1);
            g[2] = (int)q2;
        }
    } else {
        unflat(k, N, g);
    }
}
// NDIM is the grid's dimension: the neighbour arrays hold exactly the 2 NDIM
// stencil neighbours, so that they stay in registers.
template <int NDIM, typename VU, typename VR>
__device__ __forceinline__ void apply_A_node(const DevProblem& P, int64_t Ng, bool small,
                                             const float4* __restrict__ stc,
                                             const cplx<double>* __restrict__ b, const VU* __restrict__ u,
                                             VR* __restrict__ r, int nrhs, int64_t k, int c0) {
    constexpr int NB = 2 * NDIM;
    int g[3];
    unflat_nd<NDIM>(k, P.N, small, g);
    const int npt = 1 + NB;
    const float4* sk = stc + k * npt;
    // neighbour slots 2a (+1 along axis a) and 2a+1 (-1); a slot off the grid
    // (Dirichlet) is skipped
    int64_t off[NB];
    bool have[NB];
    ff cr[NB], ci[NB];
    int64_t stride = 1;
#pragma unroll
    for (int a = 0; a < NDIM; ++a) {
        have[2 * a] = g[a] + 1 < P.N[a];
        have[2 * a + 1] = g[a] > 0;
        off[2 * a] = stride;
        off[2 * a + 1] = -stride;
        const float4 qp = have[2 * a] ? sk[1 + 2 * a] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 qm = have[2 * a + 1] ? sk[2 + 2 * a] : make_float4(0.f, 0.f, 0.f, 0.f);
        cr[2 * a] = {qp.x, qp.y};
        ci[2 * a] = {qp.z, qp.w};
        cr[2 * a + 1] = {qm.x, qm.y};
        ci[2 * a + 1] = {qm.z, qm.w};
        stride *= P.N[a];
    }
    const float4 q0 = sk[0];
    const ff dr = {q0.x, q0.y}, di = {q0.z, q0.w};
    bool real = di.hi == 0.f;
#pragma unroll
    for (int i = 0; i < NB; ++i) real = real && ci[i].hi == 0.f;
    // loads of both right-hand sides first
    cff u0[kAR], un[kAR][NB], bv[kAR];
#pragma unroll
    for (int j = 0; j < kAR; ++j) {
        const int c = c0 + j < nrhs ? c0 + j : c0;
        const VU* uc = u + (int64_t)c * Ng + k;
        u0[j] = ld_c(uc);
#pragma unroll
        for (int i = 0; i < NB; ++i) un[j][i] = have[i] ? ld_c(uc + off[i]) : cff{{0.f, 0.f}, {0.f, 0.f}};
        bv[j] = b ? ld_c(b + (int64_t)c * Ng + k) : cff{{0.f, 0.f}, {0.f, 0.f}};
    }
#pragma unroll
    for (int j = 0; j < kAR; ++j) {
        if (c0 + j >= nrhs) break;
        // -(A u) accumulated onto b
        ff ar = bv[j].re, ai = bv[j].im;
        acc_mul(ar, ff_neg(dr), u0[j].re);
        acc_mul(ai, ff_neg(dr), u0[j].im);
        if (!real) {
            acc_mul(ar, di, u0[j].im);
            acc_mul(ai, ff_neg(di), u0[j].re);
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            if (!have[i]) continue;
            acc_mul(ar, ff_neg(cr[i]), un[j][i].re);
            acc_mul(ai, ff_neg(cr[i]), un[j][i].im);
            if (!real) {
                acc_mul(ar, ci[i], un[j][i].im);
                acc_mul(ai, ff_neg(ci[i]), un[j][i].re);
            }
        }
        st_c(r + (int64_t)(c0 + j) * Ng + k, cff{ar, ai});
    }
}

template <int NDIM, typename VU, typename VR>
__global__ void __launch_bounds__(256, 2)
    apply_A_kernel(DevProblem P, const float4* __restrict__ stc, const cplx<double>* __restrict__ b,
                   const VU* __restrict__ u, VR* __restrict__ r, int nrhs) {
    const int64_t Ng = (int64_t)P.N[0] * P.N[1] * P.N[2];
    const bool small = Ng <= (int64_t)UINT32_MAX;
    // node ranges along grid y, strided past the 65535-block limit
    for (int64_t kb = blockIdx.y; kb * blockDim.x < Ng; kb += gridDim.y) {
        const int64_t k = kb * blockDim.x + threadIdx.x;
        if (k < Ng) apply_A_node<NDIM>(P, Ng, small, stc, b, u, r, nrhs, k, blockIdx.x * kAR);
    }
}

template <typename VU, typename VR>
void launch_apply_A(const DevProblem& P, const float4* stc, const cplx<double>* b, const VU* u, VR* r, int nrhs,
                    cudaStream_t st) {
    const int64_t Ng = (int64_t)P.N[0] * P.N[1] * P.N[2];
    dim3 grid((nrhs + kAR - 1) / kAR, (unsigned)std::min<int64_t>((Ng + 255) / 256, 65535));
    if (P.ndim == 2)
        apply_A_kernel<2, VU, VR><<<grid, 256, 0, st>>>(P, stc, b, u, r, nrhs);
    else
        apply_A_kernel<3, VU, VR><<<grid, 256, 0, st>>>(P, stc, b, u, r, nrhs);
}
template void launch_apply_A<cplx<double>, cplx<double>>(const DevProblem&, const float4*, const cplx<double>*,
                                                         const cplx<double>*, cplx<double>*, int, cudaStream_t);
template void launch_apply_A<cplx<double>, float4>(const DevProblem&, const float4*, const cplx<double>*,
                                                   const cplx<double>*, float4*, int, cudaStream_t);
template void launch_apply_A<float4, float4>(const DevProblem&, const float4*, const cplx<double>*, const float4*,
                                             float4*, int, cudaStream_t);

// ---- batched reductions (one Krylov space per right-hand side)
constexpr int DOT_NT = 256;

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

// ---- fused multi-vector kernels of classical Gram-Schmidt: one pass over w
// and every V_i (V given as a device array of pointers to float-float vectors)

// NVB vectors per block (a compile-time count, so that the per-vector
// accumulators take only the registers they need); block z of the launch takes
// V_{ibase + z NVB} ... V_{ibase + z NVB + NVB - 1}.
template <int NVB>
__global__ void __launch_bounds__(DOT_NT, 2) mdots_partial_kernel(const float4* const* __restrict__ V, int ibase,
                                                                   const float4* __restrict__ w, int64_t n,
                                                                   int nrhs, cplx<double>* partial, int nblk) {
    __shared__ ff sr[NVB][DOT_NT / 32], si[NVB][DOT_NT / 32];
    __shared__ const float4* svp[NVB];
    const int blk = blockIdx.x, c = blockIdx.y, i0 = ibase + (int)blockIdx.z * NVB;
    constexpr int nvb = NVB;
    const int64_t chunk = (n + nblk - 1) / nblk;
    const int64_t k0 = (int64_t)blk * chunk, k1 = min(n, k0 + chunk);
    const float4* wc = w + (int64_t)c * n;
    if ((int)threadIdx.x < nvb) svp[threadIdx.x] = V[i0 + threadIdx.x] + (int64_t)c * n;
    __syncthreads();
    ff ar[NVB], ai[NVB];
#pragma unroll
    for (int i = 0; i < NVB; ++i) ar[i] = ai[i] = ff{0.f, 0.f};
    for (int64_t k = k0 + threadIdx.x; k < k1; k += DOT_NT) {
        const cff bw = ld_c(wc + k);
        cff av[NVB];
#pragma unroll
        for (int i = 0; i < NVB; ++i) av[i] = ld_c(svp[i] + k);  // vector pointers from shared memory
#pragma unroll
        for (int i = 0; i < NVB; ++i) {
            // conj(v) w = (vr br + vi bi) + i (vr bi - vi br)
            acc_mul(ar[i], av[i].re, bw.re);
            acc_mul(ar[i], av[i].im, bw.im);
            acc_mul(ai[i], av[i].re, bw.im);
            acc_mul(ai[i], ff_neg(av[i].im), bw.re);
        }
    }
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NVB; ++i) {
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
    if ((int)threadIdx.x < nvb) {
        const int i = threadIdx.x;
        ff r = {0.f, 0.f}, im = {0.f, 0.f};
        for (int q = 0; q < DOT_NT / 32; ++q) {
            r = ff_sum(r, sr[i][q]);
            im = ff_sum(im, si[i][q]);
        }
        partial[((int64_t)(i0 + i) * nrhs + c) * nblk + blk] = mk<double>(join_d(r), join_d(im));
    }
}

// squared norms |v[c]|^2 into out[c] (imaginary part 0), float-float; two
// entries per thread and step, their loads issued together
template <typename VV>
__global__ void norms_partial_kernel(const VV* __restrict__ v, int64_t n, cplx<double>* partial, int nblk) {
    __shared__ ff sr[DOT_NT / 32];
    const int blk = blockIdx.x, c = blockIdx.y;
    const int64_t chunk = (n + nblk - 1) / nblk;
    const int64_t k0 = (int64_t)blk * chunk, k1 = min(n, k0 + chunk);
    const VV* vc = v + (int64_t)c * n;
    ff a = {0.f, 0.f}, a2 = {0.f, 0.f};
    for (int64_t k = k0 + threadIdx.x; k < k1; k += 2 * DOT_NT) {
        const bool two = k + DOT_NT < k1;
        const cff x = ld_c(vc + k);
        const cff y = two ? ld_c(vc + k + DOT_NT) : cff{{0.f, 0.f}, {0.f, 0.f}};
        acc_mul(a, x.re, x.re);
        acc_mul(a, x.im, x.im);
        acc_mul(a2, y.re, y.re);
        acc_mul(a2, y.im, y.im);
    }
    a = ff_sum(a, a2);
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

template <typename VV>
void launch_norms2(const VV* v, int64_t n, int nrhs, cplx<double>* out, cplx<double>* partial, int nblk,
                   cudaStream_t st) {
    dim3 grid(nblk, nrhs);
    norms_partial_kernel<VV><<<grid, DOT_NT, 0, st>>>(v, n, partial, nblk);
    dots_final_kernel<<<(nrhs + 127) / 128, 128, 0, st>>>(partial, nblk, nrhs, out);
}
template void launch_norms2<cplx<double>>(const cplx<double>*, int64_t, int, cplx<double>*, cplx<double>*, int,
                                          cudaStream_t);
template void launch_norms2<float4>(const float4*, int64_t, int, cplx<double>*, cplx<double>*, int,
                                    cudaStream_t);

int mdots_launches(int nv) { return (nv >= 8 ? 1 : 0) + (nv % 8 ? 1 : 0) + 1; }

void launch_mdots(const float4* const* V, int nv, const float4* w, int64_t n, int nrhs, cplx<double>* out,
                  cplx<double>* partial, int nblk, cudaStream_t st) {
    // groups of 8 vectors in one launch, the rest in a second
    const int full = nv / 8, rest = nv % 8;
    if (full > 0)
        mdots_partial_kernel<8><<<dim3(nblk, nrhs, full), DOT_NT, 0, st>>>(V, 0, w, n, nrhs, partial, nblk);
    const dim3 g1(nblk, nrhs, 1);
    const int ib = full * 8;
    switch (rest) {
        case 1: mdots_partial_kernel<1><<<g1, DOT_NT, 0, st>>>(V, ib, w, n, nrhs, partial, nblk); break;
        case 2: mdots_partial_kernel<2><<<g1, DOT_NT, 0, st>>>(V, ib, w, n, nrhs, partial, nblk); break;
        case 3: mdots_partial_kernel<3><<<g1, DOT_NT, 0, st>>>(V, ib, w, n, nrhs, partial, nblk); break;
        case 4: mdots_partial_kernel<4><<<g1, DOT_NT, 0, st>>>(V, ib, w, n, nrhs, partial, nblk); break;
        case 5: mdots_partial_kernel<5><<<g1, DOT_NT, 0, st>>>(V, ib, w, n, nrhs, partial, nblk); break;
        case 6: mdots_partial_kernel<6><<<g1, DOT_NT, 0, st>>>(V, ib, w, n, nrhs, partial, nblk); break;
        case 7: mdots_partial_kernel<7><<<g1, DOT_NT, 0, st>>>(V, ib, w, n, nrhs, partial, nblk); break;
        default: break;
    }
    int count = nv * nrhs;
    dots_final_kernel<<<(count + 127) / 128, 128, 0, st>>>(partial, nblk, count, out);
}

// w[c] += sign * sum_i coef[i*nrhs+c] V_i[c], accumulated in float-float; w is
// a float-float work vector (Gram-Schmidt) or the complex128 solution (its
// update); the block's coefficients (one right-hand side per block row) are
// split once into shared memory
template <typename VW>
__global__ void mcombo_kernel(VW* w, const float4* const* __restrict__ V, int nv,
                              const cplx<double>* __restrict__ coef, int64_t n, int nrhs, double sign) {
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
    const cff w0 = ld_c(w + (int64_t)c * n + k);
    ff ar = w0.re, ai = w0.im;
    for (int i = 0; i < nv; ++i) {
        const ff cr = scr[i], ci = sci[i];
        const cff v = ld_c(V[i] + (int64_t)c * n + k);
        // (cr + i ci)(vr + i vi)
        acc_mul(ar, cr, v.re);
        acc_mul(ar, ff_neg(ci), v.im);
        acc_mul(ai, cr, v.im);
        acc_mul(ai, ci, v.re);
    }
    st_c(w + (int64_t)c * n + k, cff{ar, ai});
}

template <typename VW>
void launch_mcombo(VW* w, const float4* const* V, int nv, const cplx<double>* coef, int64_t n, int nrhs,
                   double sign, cudaStream_t st) {
    dim3 grid((unsigned)((n + 255) / 256), nrhs);
    mcombo_kernel<VW><<<grid, 256, 0, st>>>(w, V, nv, coef, n, nrhs, sign);
}
template void launch_mcombo<float4>(float4*, const float4* const*, int, const cplx<double>*, int64_t, int, double,
                                    cudaStream_t);
template void launch_mcombo<cplx<double>>(cplx<double>*, const float4* const*, int, const cplx<double>*, int64_t,
                                          int, double, cudaStream_t);

// w[c] += sum_i coef[i*nrhs+c] U_i[c] in float-float, fused with the reduction
// the next Gram-Schmidt step needs of the updated w: its dots <U_i[c], w[c]>
// with every U_i (want_dots) or its squared norm (into slot 0).  One pass over
// w and the U_i (nv <= 8, one right-hand side per block row, a fixed chunk
// per block as in the dot kernels); the dots are taken of w as stored.  NV
// and WANT_DOTS are compile-time, so that the per-vector values and
// accumulators take only the registers they need.
template <int NV, bool WANT_DOTS>
__global__ void __launch_bounds__(DOT_NT, 2) combo_dots_kernel(float4* w, const float4* const* __restrict__ U,
                                  const cplx<double>* __restrict__ coef, int64_t n, int nrhs,
                                  cplx<double>* partial, int nblk) {
    constexpr int nv = NV;
    constexpr bool want_dots = WANT_DOTS;
    constexpr int NA = WANT_DOTS ? NV : 1;  // accumulators: the dots, or the norm
    __shared__ ff scr[NV], sci[NV];
    __shared__ const float4* sup[NV];
    __shared__ ff sr[NA][DOT_NT / 32], si[NA][DOT_NT / 32];
    const int blk = blockIdx.x, c = blockIdx.y;
    if ((int)threadIdx.x < nv) {
        const cplx<double> a = coef[threadIdx.x * nrhs + c];
        scr[threadIdx.x] = split_d(a.re);
        sci[threadIdx.x] = split_d(a.im);
        sup[threadIdx.x] = U[threadIdx.x] + (int64_t)c * n;
    }
    __syncthreads();
    const int64_t chunk = (n + nblk - 1) / nblk;
    const int64_t k0 = (int64_t)blk * chunk, k1 = min(n, k0 + chunk);
    float4* wc = w + (int64_t)c * n;
    ff dr[NA], di[NA];
#pragma unroll
    for (int i = 0; i < NA; ++i) dr[i] = di[i] = ff{0.f, 0.f};
    for (int64_t k = k0 + threadIdx.x; k < k1; k += DOT_NT) {
        const cff w0 = ld_c(wc + k);
        cff uv[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) uv[i] = ld_c(sup[i] + k);  // vector pointers from shared memory
        ff ar = w0.re, ai = w0.im;
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            // (cr + i ci)(ur + i ui), the coefficients read from shared memory
            const ff cr = scr[i], ci = sci[i];
            acc_mul(ar, cr, uv[i].re);
            acc_mul(ar, ff_neg(ci), uv[i].im);
            acc_mul(ai, cr, uv[i].im);
            acc_mul(ai, ci, uv[i].re);
        }
        const cff wn = {ff_norm(ar), ff_norm(ai)};
        wc[k] = make_float4(wn.re.hi, wn.re.lo, wn.im.hi, wn.im.lo);
        if (want_dots) {
#pragma unroll
            for (int i = 0; i < NA; ++i) {
                // conj(u) w = (ur wr + ui wi) + i (ur wi - ui wr)
                acc_mul(dr[i], uv[i].re, wn.re);
                acc_mul(dr[i], uv[i].im, wn.im);
                acc_mul(di[i], uv[i].re, wn.im);
                acc_mul(di[i], ff_neg(uv[i].im), wn.re);
            }
        } else {
            acc_mul(dr[0], wn.re, wn.re);
            acc_mul(dr[0], wn.im, wn.im);
        }
    }
    constexpr int nout = NA;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NA; ++i) {
        for (int o = 16; o > 0; o >>= 1) {
            dr[i] = ff_sum(dr[i], shfl_down_ff(dr[i], o));
            di[i] = ff_sum(di[i], shfl_down_ff(di[i], o));
        }
        if (lane == 0) {
            sr[i][wp] = dr[i];
            si[i][wp] = di[i];
        }
    }
    __syncthreads();
    if ((int)threadIdx.x < nout) {
        const int i = threadIdx.x;
        ff r = {0.f, 0.f}, im = {0.f, 0.f};
        for (int q = 0; q < DOT_NT / 32; ++q) {
            r = ff_sum(r, sr[i][q]);
            im = ff_sum(im, si[i][q]);
        }
        partial[((int64_t)i * nrhs + c) * nblk + blk] = mk<double>(join_d(r), join_d(im));
    }
}

template <int NV>
static void launch_combo_dots_nv(float4* w, const float4* const* U, const cplx<double>* coef, int64_t n, int nrhs,
                                 bool want_dots, cplx<double>* partial, int nblk, cudaStream_t st) {
    const dim3 grid(nblk, nrhs);
    if (want_dots)
        combo_dots_kernel<NV, true><<<grid, DOT_NT, 0, st>>>(w, U, coef, n, nrhs, partial, nblk);
    else
        combo_dots_kernel<NV, false><<<grid, DOT_NT, 0, st>>>(w, U, coef, n, nrhs, partial, nblk);
}

cudaError_t launch_combo_dots(float4* w, const float4* const* U, int nv, const cplx<double>* coef, int64_t n,
                              int nrhs, bool want_dots, cplx<double>* out, cplx<double>* partial, int nblk,
                              cudaStream_t st) {
    switch (nv) {
        case 1: launch_combo_dots_nv<1>(w, U, coef, n, nrhs, want_dots, partial, nblk, st); break;
        case 2: launch_combo_dots_nv<2>(w, U, coef, n, nrhs, want_dots, partial, nblk, st); break;
        case 3: launch_combo_dots_nv<3>(w, U, coef, n, nrhs, want_dots, partial, nblk, st); break;
        case 4: launch_combo_dots_nv<4>(w, U, coef, n, nrhs, want_dots, partial, nblk, st); break;
        case 5: launch_combo_dots_nv<5>(w, U, coef, n, nrhs, want_dots, partial, nblk, st); break;
        case 6: launch_combo_dots_nv<6>(w, U, coef, n, nrhs, want_dots, partial, nblk, st); break;
        case 7: launch_combo_dots_nv<7>(w, U, coef, n, nrhs, want_dots, partial, nblk, st); break;
        case 8: launch_combo_dots_nv<8>(w, U, coef, n, nrhs, want_dots, partial, nblk, st); break;
        default: return cudaErrorInvalidValue;  // nv outside 1 .. kComboDotsMax: nothing launched
    }
    const int count = (want_dots ? nv : 1) * nrhs;
    dots_final_kernel<<<(count + 127) / 128, 128, 0, st>>>(partial, nblk, count, out);
    return cudaSuccess;
}

__global__ void conj_kernel(cplx<double>* v, int64_t count) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < count) v[k].im = -v[k].im;
}

void launch_conj(cplx<double>* v, int64_t count, cudaStream_t st) {
    conj_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(v, count);
}

// w = b in float-float form (the residual b - A x of a zero x): one entry per
// thread, grid-strided.
__global__ void to_ff_kernel(const cplx<double>* __restrict__ b, float4* __restrict__ w, int64_t count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        st_c(w + i, ld_c(b + i));
}

void launch_to_ff(const cplx<double>* b, float4* w, int64_t count, cudaStream_t st) {
    const int64_t blocks = std::min<int64_t>((count + 255) / 256, 152 * 16);
    to_ff_kernel<<<(unsigned)blocks, 256, 0, st>>>(b, w, count);
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
