// Subdomain solves on the 5th-generation tensor cores: tcgen05.mma (kind::tf32,
// and kind::f16 with power-of-two scaled operands) with TMEM accumulators,
// operands in shared memory fed by the bulk-copy engine.  Two kernels:
//   * solve_twist_kernel (the default): the twisted factors, solved from both
//     ends toward the middle line by the two CTAs of a cluster, each holding
//     all rows of the block -- described before its definition below;
//   * solve_umma_kernel (one-ended): the block rows split over the CTAs of a
//     cluster, the next right-hand side exchanged every step -- described here.
//
// Recurrence (block-Thomas, k_factor.cu): forward y_j = D_j (b_j - a_j y_{j-1}),
// backward u_j = y_j - D_j (c_j u_{j+1}).  Each block product D_j R is one real
// GEMM  Y[M=n rows][N=2*PG] = A[M][K] B[K][N]  with
//   K index k = 2q + part:   A[p][2q+part] = part ? Im D(p,q) : Re D(p,q)
//   N index n = 2c + w:      B[2q][2c] = Re r, B[2q+1][2c] = -Im r,
//                            B[2q][2c+1] = Im r, B[2q+1][2c+1] = Re r
// so Y[p][2c] = Re y_pc and Y[p][2c+1] = Im y_pc.
//
// Layouts (all K-major with the 128-byte swizzle: rows of 32 TF32 values, the
// 16-byte chunk c of row r stored at chunk c ^ (r % 8), 8-row groups 1024 B apart):
//   * A: the factors are repacked once (repack_umma_kernel) into the exact
//     shared-memory image, [line][K chunk of 32][CTA of the cluster][R rows x 128 B].
//     The block rows are split evenly over the CR CTAs of a cluster (R = n/CR
//     rounded up to 8 rows), so each K chunk of each CTA is one contiguous span
//     for cp.async.bulk and a CTA streams only R*128 bytes per chunk: the ring
//     then holds more than one line step, and the next step's operand arrives
//     while the current one is multiplied.
//   * B: built in shared memory by the epilogue threads, [K chunk][N rows][128 B].
//
// Roles (one CTA per (task, panel of PG right-hand sides, R-row slice of the
// block); the CR slices of a block form a thread-block cluster, N = 2 PG;
// each MMA has M = 128, and accumulator rows R..127 are ignored):
//   warps 0-3   epilogue: thread = one block row p; reads its row of the
//               accumulator from TMEM (tcgen05.ld), stores y or u, and writes
//               row p of the next B into its own CTA; one thread then pushes
//               the CTA's rows of B to the peer CTA with one bulk copy (DSMEM)
//   warps 4-7   producers: lane 0 of warp 4+q bulk-copies the K chunks at
//               stream positions q, q+4, ... of this CTA's slice of A (own
//               rows' chunks first) into sub-ring q of the ring
//   warps 8-11  lane 0 of warp 8+q issues the MMAs of those chunks into its
//               own accumulator and commits; warp 8 also allocates TMEM
// Handshakes are mbarriers: full/empty per stage (TMA bytes / tcgen05.commit),
// acc_full per step (tcgen05.commit), b_local per step (own rows of B
// written: the K chunks of this CTA's rows are multiplied at once) and
// b_remote per step (the peer's rows have arrived: armed by this CTA with
// the bytes it expects, completed by the peer's bulk copy), so the exchange
// overlaps the MMAs of the CTA's own chunks.
// Every wait is bounded; on expiry the CTA raises the device error word, each
// role leaves its loop, outstanding copies and MMAs are drained (bounded),
// the two CTAs drain the bulk copies between them, and TMEM is freed before
// the CTA exits.
#include <algorithm>

#include <cuda_fp16.h>

#include "helm_internal.h"
#include "tc_util.cuh"

namespace helm {

using namespace tc;

namespace {

constexpr uint32_t kWait = kDrainPolls;
constexpr int kChunkK = 32;        // K values per 128-byte row
constexpr int kTileBytes = 128 * 128;  // 128 rows x 128 B

}  // namespace

// Block rows held by each of the CR CTAs of a cluster: an even split rounded
// up to 16 rows (whole 8-row swizzle groups of A, and whole 32-value K chunks
// of B: 2 values per row), at most 128 = the MMA's M when n <= 128 CR.
__host__ __device__ inline int umma_rows(int n, int CR) { return (((n + CR - 1) / CR) + 15) & ~15; }

// Bytes of one line's repacked A for a block of n rows split over CR CTAs
// (every subdomain of a context uses the same CR):
// ceil(2*roundup4(n)/32) K chunks x CR slices x R rows x 128 B.
__host__ __device__ inline int64_t umma_line_bytes(int n, int CR, int* nkc) {
    const int n4 = (n + 3) & ~3;
    const int kc = (2 * n4 + kChunkK - 1) / kChunkK;
    if (nkc) *nkc = kc;
    return (int64_t)kc * CR * umma_rows(n, CR) * 128;
}

// FP16 image for the twisted solve (one slice, all rows): K chunks of 64
// values (128 bytes of halves per row), R = roundup16(n) rows.
__host__ __device__ inline int64_t umma_line_bytes16(int n, int* nkc) {
    const int n4 = (n + 3) & ~3;
    const int kc = (2 * n4 + 63) / 64;
    if (nkc) *nkc = kc;
    return (int64_t)kc * umma_rows(n, 1) * 128;
}

// Repack the column-major factors of every subdomain (k_factor.cu layout) into
// the swizzled tile image, rounding to TF32.  One thread per output float.
__global__ void repack_umma_kernel(const SubDesc* __restrict__ subs, const float* __restrict__ fac,
                                   const float* __restrict__ fac2, const int64_t* __restrict__ dst_off,
                                   float* dst, int sub, int cr) {
    const SubDesc& S = subs[sub];
    int nkc;
    const int64_t lb = umma_line_bytes(S.nblk, cr, &nkc) / 4;  // floats per line
    const int R = umma_rows(S.nblk, cr);
    const int64_t total = lb * S.nlines;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int j = (int)(i / lb);
    int64_t rem = i % lb;
    const int kc = (int)(rem / (cr * R * 32));
    rem %= (cr * R * 32);
    const int slice = (int)(rem / (R * 32));
    const int off = (int)(rem % (R * 32));  // float offset in the slice image
    const int r = off / 32;                 // row in the slice
    const int pos = off % 32;               // float position within the 128-byte row
    const int chunk = (pos / 4) ^ (r % 8);
    const int kk = chunk * 4 + (pos % 4);  // logical K within the chunk
    const int p = slice * R + r;
    const int k = kc * kChunkK + kk;
    const int q = k >> 1, part = k & 1;
    float v = 0.f;
    if (p < S.nblk && q < S.nblk) {
        // lines from nlines/2 on come from the twisted factors when there are any
        const float* src = (fac2 && j >= S.nlines / 2) ? fac2 : fac;
        const float* D = src + S.fac_off + (int64_t)j * 2 * S.nbp * S.nbp;
        v = D[(int64_t)q * 2 * S.nbp + part * S.nbp + p];
    }
    dst[dst_off[sub] / 4 + i] = __uint_as_float(to_tf32(v));  // dst_off in bytes
}

// Per-line power-of-two scale of the FP16 factor image: ascale[inva_off + j]
// = 13 - floor(log2 max|Re, Im D_j|), so the largest entry of a line lands in
// [2^13, 2^14) (FP16 holds up to 65504).  One block per (subdomain, line);
// lines from nlines/2 on read the twisted factors.
__global__ void line_scale_kernel(const SubDesc* __restrict__ subs, const float* __restrict__ fac,
                                  const float* __restrict__ fac2, int* ascale) {
    const SubDesc& S = subs[blockIdx.x];
    const int j = blockIdx.y;
    if (j >= S.nlines) return;
    const float* src = (fac2 && j >= S.nlines / 2) ? fac2 : fac;
    const float* D = src + S.fac_off + (int64_t)j * 2 * S.nbp * S.nbp;
    const int n = S.nblk;
    uint32_t mx = 0;
    for (int64_t e = threadIdx.x; e < (int64_t)n * 2 * n; e += blockDim.x) {
        const int q = (int)(e / (2 * n)), r = (int)(e % (2 * n));
        const int part = r / n, p = r % n;
        const float v = fabsf(D[(int64_t)q * 2 * S.nbp + part * S.nbp + p]);
        mx = max(mx, __float_as_uint(v));  // non-negative floats order as their bits
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    __shared__ uint32_t wm[32];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = max(mx, wm[w]);
        mx = max(mx, wm[0]);
        int sc = 0;
        if (mx != 0 && mx < 0x7F800000u) {
            const int e = (int)((mx >> 23) & 0xFF) - 127;  // floor(log2) of a normal float
            sc = 13 - e;
            sc = sc < -60 ? -60 : (sc > 60 ? 60 : sc);
        }
        ascale[S.inva_off + j] = sc;
    }
}

// FP16 image of the factors for the twisted solve: [line][K chunk of 64][R rows x
// 128 B], 128-byte swizzle, each line scaled by 2^ascale; one thread per half.
__global__ void repack_f16_kernel(const SubDesc* __restrict__ subs, const float* __restrict__ fac,
                                  const float* __restrict__ fac2, const int* __restrict__ ascale,
                                  const int64_t* __restrict__ dst_off, __half* dst, int sub) {
    const SubDesc& S = subs[sub];
    int nkc;
    const int64_t lb = umma_line_bytes16(S.nblk, &nkc) / 2;  // halves per line
    const int R = umma_rows(S.nblk, 1);
    const int64_t total = lb * S.nlines;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int j = (int)(i / lb);
    const int64_t rem = i % lb;
    const int kc = (int)(rem / (R * 64));
    const int off = (int)(rem % (R * 64));
    const int r = off / 64, pos = off % 64;  // row; half position within the 128-byte row
    const int unit = (pos / 8) ^ (r % 8);
    const int k = kc * 64 + unit * 8 + (pos % 8);
    const int q = k >> 1, part = k & 1;
    float v = 0.f;
    if (r < S.nblk && q < S.nblk) {
        const float* src = (fac2 && j >= S.nlines / 2) ? fac2 : fac;
        const float* D = src + S.fac_off + (int64_t)j * 2 * S.nbp * S.nbp;
        v = D[(int64_t)q * 2 * S.nbp + part * S.nbp + r] * pow2f(ascale[S.inva_off + j]);
    }
    dst[dst_off[sub] / 2 + i] = __float2half_rn(v);  // dst_off in bytes
}


// One CTA per (task, panel of PG right-hand sides, R-row slice of the block);
// the slices of one block form a cluster of CR (1 or 2).  Each CTA streams and
// multiplies only its own rows of D_j, holds the whole K extent of B, and its
// epilogue writes the B rows of its block rows into both CTAs of the cluster.
// B is double-buffered: a peer may be one step ahead.
constexpr int kIssuers = 4;  // MMA-issuing warps; K chunks are dealt round-robin to them
// One bulk-copy producer warp per issuer: a thread issues one cp.async.bulk
// every ~350 ns whatever its size, so a single producer of 12 KB chunks
// supplies only ~35 GB/s to its SM, and four supply four times that.
constexpr int kWarpEpi = 4, kWarpProd = kWarpEpi, kWarpIss = kWarpProd + kIssuers;
constexpr int kThreads = 32 * (kWarpIss + kIssuers);

template <int PG>
__global__ void __launch_bounds__(kThreads) solve_umma_kernel(
    const Task* __restrict__ tasks, const SubDesc* __restrict__ subs, int nrhs, int CR,
    const float* __restrict__ afac, const int64_t* __restrict__ afac_off,
    const cplx<float>* __restrict__ Pv, const cplx<float>* __restrict__ inva, cplx<float>* buf,
    const cplx<float>* __restrict__ bsrc, int64_t rstride, int nstage, uint32_t ring_bytes, DevStatus ds) {
    constexpr int kN = 2 * PG;              // real columns
    constexpr int kBChunkBytes = kN * 128;  // B rows of one K chunk
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t rank = CR > 1 ? cluster_rank() : 0;
    const Task tk = tasks[blockIdx.x / CR];
    const SubDesc& S = subs[tk.sub];
    const int n = S.nblk, nl = S.nlines;
    int nkc;
    const int64_t line_bytes = umma_line_bytes(n, CR, &nkc);
    const int R = umma_rows(n, CR);                  // block rows of this CTA
    const uint32_t stage_bytes = (uint32_t)R * 128;  // one K chunk of them
    const int NS = nstage;
    const uint32_t bbuf_bytes = (uint32_t)(nkc * kBChunkBytes);

    // shared layout (1024-aligned): ring | B[2] | barriers | tmem slot | flag.
    // The ring holds NS stages of stage_bytes plus a tail, ring_bytes in all
    // (>= NS*stage_bytes + 16 KB - stage_bytes), so the 128-row operand an MMA
    // reads from the last stage stays inside the ring; rows R..127 of a stage
    // are whatever follows it and only feed accumulator rows that are ignored.
    const uint32_t base = (su32(smem_raw) + 1023u) & ~1023u;
    unsigned char* gbase = smem_raw + (base - su32(smem_raw));
    const uint32_t stage0 = base;
    const uint32_t b0 = stage0 + ring_bytes;
    float* bgen = reinterpret_cast<float*>(gbase + ring_bytes);
    const uint32_t bars = b0 + 2 * bbuf_bytes;
    uint64_t* bars_g = reinterpret_cast<uint64_t*>(gbase + ring_bytes + 2 * bbuf_bytes);
    // The ring is split into kIssuers sub-rings of NQ stages, one per issuer
    // (stage q*NQ + k): the chunk at stream position li of a line goes to
    // issuer li % kIssuers, which consumes its chunks in stream order, so every
    // stage has one producer and one consumer in order and a parity wait on it
    // always refers to the expected phase, however the copies complete.
    const int NQ = NS / kIssuers;
    auto full = [&](int s) { return bars + 8u * s; };
    auto empty = [&](int s) { return bars + 8u * (NS + s); };
    const uint32_t acc_full = bars + 8u * (2 * NS);
    // B of step s is double-buffered (buffer s & 1) and announced by two
    // barriers of parity s & 1: b_local when this CTA's own rows are written
    // (their K chunks can be multiplied at once), b_remote when every peer's
    // rows have arrived.  Consecutive steps never share a phase (a peer may
    // announce step s+1 before this CTA has consumed step s).
    auto b_local = [&](int step) { return bars + 8u * (2 * NS + 1 + (step & 1)); };
    auto b_remote = [&](int step) { return bars + 8u * (2 * NS + 3 + (step & 1)); };
    const uint32_t drain = bars + 8u * (2 * NS + 5);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars_g + 2 * NS + 6);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    int* rem_done = reinterpret_cast<int*>(tmem_slot + 2);  // steps whose b_remote phase an issuer passed
    volatile int* cnt_in = reinterpret_cast<volatile int*>(tmem_slot + 3);  // copies the peer sent (exit)
    volatile int* cnt_out = reinterpret_cast<volatile int*>(tmem_slot + 4);  // copies this CTA sent

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nsteps = 2 * nl - 1;
    // K chunks in the order this CTA streams and multiplies them: first the
    // nloc chunks of its own block rows (B rows 2p, 2p+1 of rows p it owns),
    // then the peers' chunks, which wait for the exchange
    const int nkr = R / 16;  // K chunks per CTA's rows
    int nloc = nkc - (int)rank * nkr;
    nloc = nloc < 0 ? 0 : (nloc > nkr ? nkr : nloc);
    auto chunk_at = [&](int li) { return (li + (int)rank * nkr) % nkc; };
    // bytes of B rows this CTA sends to / receives from the peer per step
    const uint32_t peer = rank ^ 1u;  // the other CTA of a 2-CTA cluster
    int nloc_peer = nkc - (int)peer * nkr;
    nloc_peer = nloc_peer < 0 ? 0 : (nloc_peer > nkr ? nkr : nloc_peer);
    const uint32_t own_bytes = (uint32_t)nloc * kBChunkBytes;
    const uint32_t peer_bytes = (uint32_t)nloc_peer * kBChunkBytes;
    // one accumulator of kN columns per issuer
    constexpr uint32_t kCols = kIssuers * kN <= 32 ? 32 : kIssuers * kN <= 64 ? 64 :
                               kIssuers * kN <= 128 ? 128 : 256;

    if (tid == 0) {
        *abort_flag = 0;
        *rem_done = 0;
        *cnt_in = 0;
        *cnt_out = 0;
        for (int s = 0; s < NS; ++s) {
            mb_init(full(s), 1);
            mb_init(empty(s), 1);
        }
        mb_init(acc_full, kIssuers);
        mb_init(b_local(0), 1);  // this CTA's epilogue
        mb_init(b_local(1), 1);
        mb_init(b_remote(0), 1);  // this CTA's epilogue arms it for the peer's rows (unused if CR = 1)
        mb_init(b_remote(1), 1);
        mb_init(drain, kIssuers);  // completes once every issuer's MMAs have
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (uint32_t i = tid; i < 2 * bbuf_bytes / 4; i += blockDim.x) bgen[i] = 0.f;
    {
        float* sg = reinterpret_cast<float*>(gbase);
        for (uint32_t i = tid; i < ring_bytes / 4; i += blockDim.x) sg[i] = 0.f;
    }
    if (warp == kWarpIss) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    if (CR > 1) cluster_sync();  // peers' barriers are initialised before any remote arrive
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp >= kWarpProd && warp < kWarpProd + kIssuers) {
        // ====================================================== producers
        // producer p fills sub-ring p with the chunks at stream positions
        // p, p + kIssuers, ... of every line, in order
        const int pq = warp - kWarpProd;
        if (lane == 0) {
            const char* abase = reinterpret_cast<const char*>(afac) + afac_off[tk.sub];
            int k = 0;  // chunks put into this sub-ring so far
            for (int step = 0; step < nsteps && !*abort_flag; ++step) {
                const int j = step < nl ? step : 2 * nl - 2 - step;
                for (int li = pq; li < nkc; li += kIssuers) {
                    const int s = pq * NQ + k % NQ;
                    if (k >= NQ && !mb_wait(empty(s), (uint32_t)(((k / NQ) - 1) & 1), ds.polls)) {
                        atomicExch(ds.err, 2);
                        *abort_flag = 1;
                    }
                    if (*abort_flag) break;
                    const int64_t chunk_off = ((int64_t)chunk_at(li) * CR + rank) * stage_bytes;
                    mb_expect_tx(full(s), stage_bytes);
                    bulk_g2s(stage0 + s * stage_bytes, abase + (int64_t)j * line_bytes + chunk_off, stage_bytes,
                             full(s));
                    ++k;
                }
            }
            // drain: every issued copy lands before the shared memory is released
            for (int kk = (k > NQ ? k - NQ : 0); kk < k; ++kk)
                mb_wait(full(pq * NQ + kk % NQ), (uint32_t)((kk / NQ) & 1), kWait);
        }
    } else if (warp >= kWarpIss && warp < kWarpIss + kIssuers) {
        // ====================================================== MMA issuers
        // issuer q takes the chunks at positions q, q + kIssuers, ... of the
        // stream order of every line into its own accumulator (columns q*kN
        // ...), so the per-instruction issue latency overlaps across warps
        const int q = warp - kWarpIss;
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_tf32(128, kN);
            const uint32_t dacc = tmem + (uint32_t)(q * kN);
            int k = 0;  // chunks of this issuer so far (its sub-ring sequence)
            for (int step = 0; step < nsteps && !*abort_flag; ++step) {
                if (!mb_wait(b_local(step), (uint32_t)((step >> 1) & 1), ds.polls)) {
                    atomicExch(ds.err, 2);
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                const uint64_t bdesc0 = desc_sw128(b0 + (step & 1) * bbuf_bytes);
                bool first = true, peers_in = CR == 1;
                for (int li = q; li < nkc; li += kIssuers) {
                    if (li >= nloc && !peers_in) {
                        if (!mb_wait(b_remote(step), (uint32_t)((step >> 1) & 1), ds.polls)) {
                            atomicExch(ds.err, 2);
                            *abort_flag = 1;
                            break;
                        }
                        tc_fence_after();
                        peers_in = true;
                        atomicMax(rem_done, step + 1);
                    }
                    const int kc = chunk_at(li);
                    const int s = q * NQ + k % NQ;
                    const uint32_t par = (uint32_t)((k / NQ) & 1);
                    ++k;
                    if (!mb_wait(full(s), par, ds.polls)) {
                        atomicExch(ds.err, 2);
                        *abort_flag = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t adesc = desc_sw128(stage0 + s * stage_bytes);
                    const uint64_t bdesc = bdesc0 + (uint64_t)(kc * (kBChunkBytes >> 4));
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        umma_tf32(dacc, adesc + (uint64_t)(2 * kk), bdesc + (uint64_t)(2 * kk), idesc,
                                  (first && kk == 0) ? 0u : 1u);
                    first = false;
                    umma_commit(empty(s));
                }
                if (*abort_flag) break;
                // (an issuer without a chunk -- K shorter than kIssuers chunks -- commits
                // nothing pending; the epilogue never reads its accumulator).  An
                // issuer whose chunks are all local still waits for the peers' rows
                // of this step before committing, so that b_remote's phases are
                // consumed in step order by every issuer.
                if (!peers_in) {
                    if (!mb_wait(b_remote(step), (uint32_t)((step >> 1) & 1), ds.polls)) {
                        atomicExch(ds.err, 2);
                        *abort_flag = 1;
                        break;
                    }
                    atomicMax(rem_done, step + 1);
                }
                umma_commit(acc_full);
            }
            umma_commit(drain);
            mb_wait(drain, 0u, kWait);
        }
    } else {
        // ====================================================== epilogue (warps 0-3)
        const int lr = warp * 32 + lane;     // accumulator row (TMEM lane)
        const int p = (int)rank * R + lr;    // block row, owned if lr < R
        const bool own = lr < R;
        const bool rv = own && p < n;
        const int n4 = (n + 3) & ~3;
        const cplx<float> pvp = rv ? Pv[S.coup_off + p] : mk<float>(0, 0);
        const cplx<float>* ia = inva + S.inva_off;
        cplx<float>* V = buf + tk.buf_off;
        const int c0 = blockIdx.y * PG;
        int ncol = nrhs - c0;
        if (ncol > PG) ncol = PG;
        const int k0 = 2 * p;  // B rows k0 (Re column) and k0+1 (Im column)
        const int kcb = k0 / kChunkK, kkb = k0 % kChunkK;
        // byte offset of B[row][k0] within a buffer (k0, k0+1 adjacent)
        auto boff = [&](int row) -> uint32_t {
            const int chunk = (kkb / 4) ^ (row % 8);
            return (uint32_t)(kcb * kBChunkBytes + row * 128 + chunk * 16 + (kkb % 4) * 4);
        };
        const uint32_t peer_b = CR > 1 ? map_peer(b0, peer) : b0;
        const uint32_t peer_remote = CR > 1 ? map_peer(b_remote(0), peer) : b_remote(0);  // parity 1: +8
        // this CTA's rows of B: its nloc K chunks from chunk rank*nkr
        const uint32_t own_off = (uint32_t)((int)rank * nkr) * kBChunkBytes;
        const bool wr = own && p < n4;  // this thread writes B rows 2p, 2p+1
        // B rows k0, k0+1 of right-hand side c: row 2c holds (Re r, -Im r),
        // row 2c+1 holds (Im r, Re r); values rounded to TF32
        auto put_local = [&](int bb, const cplx<float> (&v)[PG]) {
            float* bl = reinterpret_cast<float*>(gbase + ring_bytes + (uint32_t)bb * bbuf_bytes);
#pragma unroll
            for (int c = 0; c < PG; ++c) {
                const float re = __uint_as_float(to_tf32(v[c].re)), im = __uint_as_float(to_tf32(v[c].im));
                const float nim = __uint_as_float(to_tf32(-v[c].im));
                *reinterpret_cast<float2*>(bl + boff(2 * c) / 4) = make_float2(re, nim);
                *reinterpret_cast<float2*>(bl + boff(2 * c + 1) / 4) = make_float2(im, re);
            }
        };
        // Announce the B rows of `step`: each writer orders its stores before
        // the async-proxy reads (tensor cores, bulk copy) and its TMEM loads
        // before the thread sync; after the epilogue barrier one thread
        //   * arrives on b_local: this CTA's own K chunks can be multiplied;
        //   * (2-CTA clusters) arms b_remote for the peer's rows of this step
        //     (one arrival + their bytes; they may land before or after), and
        //     pushes this CTA's rows, one contiguous run of whole K chunks,
        //     into the peer's B buffer with a bulk copy that completes on the
        //     peer's b_remote.
        // Buffer reuse is safe without further waits: the peer multiplies
        // step s only after its own step s-1, which needed this CTA's rows of
        // s-1, sent after this CTA finished multiplying s-2 -- and the same
        // chain orders this CTA's next write of a buffer after the peer has
        // received (and the copy has finished reading) its previous contents.
        auto announce = [&](int step, const cplx<float> (&v)[PG]) {
            if (wr) put_local(step & 1, v);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_fence_before();
            epi_sync();
            if (tid == 0) {
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b_local(step)) : "memory");
                if (CR > 1) {
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b_remote(step)),
                                 "r"(peer_bytes)
                                 : "memory");
                    const uint32_t off = (uint32_t)(step & 1) * bbuf_bytes + own_off;
                    if (own_bytes) bulk_s2peer(peer_b + off, b0 + off, own_bytes, peer_remote + 8u * (step & 1));
                    *cnt_out = step + 1;  // steps armed and sent
                }
            }
        };
        // operand needed after the product of step s: b_{j+1} (forward line j)
        // or y_j (backward line j); loaded one whole step ahead
        auto operand_line = [&](int step) -> int {
            if (step >= nsteps) return -1;
            if (step < nl) return step + 1 < nl ? step + 1 : -1;
            return 2 * nl - 2 - step;
        };
        const cplx<float>* Bsrc = bsrc + tk.buf_off;  // the local source b
        auto load_operand = [&](int step, cplx<float> (&dst)[PG]) {
            const int jj = operand_line(step);
            const cplx<float>* src = step < nl ? Bsrc : V;  // b_{j+1} forward, y_j backward
#pragma unroll
            for (int c = 0; c < PG; ++c)
                dst[c] = (rv && c < ncol && jj >= 0) ? src[(int64_t)(c0 + c) * rstride + (int64_t)jj * n + p]
                                                     : mk<float>(0, 0);
        };
        cplx<float> pre[PG], pre_next[PG], outv[PG], nbv[PG];
#pragma unroll
        for (int c = 0; c < PG; ++c)
            nbv[c] = (rv && c < ncol) ? Bsrc[(int64_t)(c0 + c) * rstride + p] : mk<float>(0, 0);
        load_operand(0, pre);
        announce(0, nbv);
        for (int step = 0; step < nsteps; ++step) {
            const bool fwd = step < nl;
            const int j = fwd ? step : 2 * nl - 2 - step;
            load_operand(step + 1, pre_next);
            bool bad = *abort_flag || !mb_wait(acc_full, (uint32_t)(step & 1), ds.polls);
            if (epi_any(bad)) {  // uniform over the epilogue: before the collective load and barriers
                atomicExch(ds.err, 2);
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            // sum of the issuers' partial accumulators (an issuer without a chunk --
            // K shorter than kIssuers chunks -- holds none); loads go out in groups
            // of at most 64 registers, each group waited for once
            constexpr int kGroup = kN * kIssuers <= 64 ? kIssuers : (64 / kN > 0 ? 64 / kN : 1);
            float acc[kN];
#pragma unroll
            for (int e = 0; e < kN; ++e) acc[e] = 0.f;
#pragma unroll
            for (int g0 = 0; g0 < kIssuers; g0 += kGroup) {
                uint32_t part[kGroup][kN / 16][16];
#pragma unroll
                for (int ig = 0; ig < kGroup; ++ig)
#pragma unroll
                    for (int q = 0; q < kN / 16; ++q)
                        if (g0 + ig < nkc)
                            tmem_ld16_async(tmem + ((uint32_t)(warp * 32) << 16) + (g0 + ig) * kN + 16 * q,
                                            part[ig][q]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int ig = 0; ig < kGroup; ++ig)
#pragma unroll
                    for (int q = 0; q < kN / 16; ++q) {
                        if (g0 + ig >= nkc) continue;
                        tmem_pin16(part[ig][q]);
#pragma unroll
                        for (int e = 0; e < 16; ++e) acc[16 * q + e] += __uint_as_float(part[ig][q][e]);
                    }
            }
            cplx<float> coup = mk<float>(0, 0);
            if (rv) {
                if (fwd && j + 1 < nl) coup = pvp * ia[j + 1];   // a_{j+1}
                else if (fwd) coup = pvp * ia[nl - 1];            // c_{nl-2}
                else if (j > 0) coup = pvp * ia[j];               // c_{j-1}
            }
#pragma unroll
            for (int c = 0; c < PG; ++c) {
                const cplx<float> y = mk<float>(acc[2 * c], acc[2 * c + 1]);
                outv[c] = fwd ? y : pre[c] - y;
                nbv[c] = mk<float>(0, 0);
                if (rv) nbv[c] = (fwd && j + 1 < nl) ? pre[c] - coup * outv[c] : coup * outv[c];
            }
            if (step + 1 < nsteps) announce(step + 1, nbv);
            // global stores after the release-arrive, so it does not wait for them
#pragma unroll
            for (int c = 0; c < PG; ++c) {
                if (rv && c < ncol) V[(int64_t)(c0 + c) * rstride + (int64_t)j * n + p] = outv[c];
                pre[c] = pre_next[c];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (CR > 1) {
        // Drain the bulk copies between the two CTAs before either leaves (after
        // an abort they may differ in how many steps they announced): each CTA
        // learns how many copies its peer sent, arms the phases of b_remote it
        // had not armed, and waits, in phase order, until every copy addressed
        // to it has landed; the second cluster barrier then keeps each CTA
        // resident until the copies reading its shared memory have finished.
        if (tid == 0) {
            const uint32_t dst = map_peer(su32((const void*)cnt_in), peer);
            asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(dst), "r"((uint32_t)*cnt_out) : "memory");
        }
        __syncwarp();
        cluster_sync();
        if (tid == 0) {
            const int k_in = *cnt_in, armed = *cnt_out;
            for (int st = *reinterpret_cast<volatile int*>(rem_done); st < k_in; ++st) {
                if (st >= armed)
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b_remote(st)),
                                 "r"(peer_bytes)
                                 : "memory");
                if (!mb_wait(b_remote(st), (uint32_t)((st >> 1) & 1), kWait)) {
                    atomicExch(ds.err, 2);
                    break;
                }
            }
        }
        __syncwarp();
        cluster_sync();
    }
    tc_fence_after();
    if (warp == kWarpIss)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols)
                     : "memory");
}

void launch_repack_umma(const SubDesc* subs_d, const std::vector<SubDesc>& subs_h, int mt,
                        const float* fac, const float* fac2, const int64_t* dst_off_d, float* dst,
                        cudaStream_t st) {
    for (size_t s = 0; s < subs_h.size(); ++s) {
        const int64_t floats = umma_line_bytes(subs_h[s].nblk, mt, nullptr) / 4 * subs_h[s].nlines;
        repack_umma_kernel<<<(unsigned)((floats + 255) / 256), 256, 0, st>>>(subs_d, fac, fac2, dst_off_d,
                                                                             dst, (int)s, mt);
    }
}

int umma_tiles(int nblk_max) { return (nblk_max + 127) / 128; }

int64_t umma_factor_bytes(const SubDesc& S, int mt) { return umma_line_bytes(S.nblk, mt, nullptr) * S.nlines; }

// Shared-memory plan of a launch: ring of ns stages (kIssuers sub-rings, at
// least 2 stages each, at most 32 stages) plus the 128-row tail of the last
// stage, B[2], barriers and slots, alignment.  Returns the bytes, or 0 if the
// minimum ring does not fit in a CTA's 227 KB.
static size_t umma_smem_plan(int PG, int CR, int nblk_max, int* ns_out, uint32_t* ring_out) {
    int nkc_max = 0;
    umma_line_bytes(nblk_max, CR, &nkc_max);
    const size_t sb_max = (size_t)umma_rows(nblk_max, CR) * 128;  // largest stage
    const size_t bbuf = (size_t)nkc_max * 2 * PG * 128;
    const size_t fixed = 2 * bbuf + 1024 + 1024;  // B[2]; barriers, slots; alignment
    const size_t budget = 227 * 1024;
    if (fixed + (2 * kIssuers - 1) * sb_max + kTileBytes > budget) return 0;
    int ns = (int)((budget - fixed - kTileBytes) / sb_max) + 1;
    if (ns > 32) ns = 32;  // barriers: 2 ns + 6 of 8 bytes within the 1 KB reserve
    ns -= ns % kIssuers;
    const uint32_t ring = (uint32_t)((ns - 1) * sb_max + kTileBytes);
    *ns_out = ns;
    *ring_out = ring;
    return ring + fixed;
}

template <int PG>
static void launch_pg(const Task* tasks, int ntask, const SubDesc* subs, int CR, int nblk_max,
                      int nrhs, const float* afac, const int64_t* afac_off, const cplx<float>* Pv,
                      const cplx<float>* inva, cplx<float>* buf, const cplx<float>* bsrc, int64_t rstride,
                      DevStatus ds, cudaStream_t st) {
    int ns = 0;
    uint32_t ring_bytes = 0;
    const size_t smem = umma_smem_plan(PG, CR, nblk_max, &ns, &ring_bytes);
    cudaFuncSetAttribute(solve_umma_kernel<PG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ntask * CR, (nrhs + PG - 1) / PG, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CR;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, solve_umma_kernel<PG>, tasks, subs, nrhs, CR, afac, afac_off, Pv, inva,
                       buf, bsrc, rstride, ns, ring_bytes, ds);
}

bool umma_supported(int nblk_max) {
    int ns;
    uint32_t ring;
    return umma_tiles(nblk_max) <= 2 && umma_smem_plan(8, umma_tiles(nblk_max), nblk_max, &ns, &ring) != 0;
}

void launch_solve_umma(const Task* tasks, int ntask, const SubDesc* subs, int nblk_max, int nrhs,
                       int panel, const float* afac, const int64_t* afac_off,
                       const cplx<float>* Pv, const cplx<float>* inva, cplx<float>* buf,
                       const cplx<float>* bsrc, int64_t rstride, DevStatus ds, cudaStream_t st) {
    if (ntask == 0) return;
    const int CR = umma_tiles(nblk_max);  // cluster of ceil(n / 128) CTAs, rows split evenly
    int ns;
    uint32_t ring;
    // the widest panel (up to the one asked for) whose shared-memory plan fits
    int pg = panel >= 32 ? 32 : panel >= 16 ? 16 : 8;
    while (pg > 8 && umma_smem_plan(pg, CR, nblk_max, &ns, &ring) == 0) pg /= 2;
#define HELM_UMMA(PG_) \
    launch_pg<PG_>(tasks, ntask, subs, CR, nblk_max, nrhs, afac, afac_off, Pv, inva, buf, bsrc, rstride, ds, st)
    if (pg == 32) HELM_UMMA(32); else if (pg == 16) HELM_UMMA(16); else HELM_UMMA(8);
#undef HELM_UMMA
}


// ============================================================================
// Twisted (two-ended) block solve on the tensor cores.
//
// With the twisted factors (k_factor.cu: D_j = S_j^{-1} for lines j < mid,
// F = M^{-1} at mid = nl/2, E_j = T_j^{-1} for j > mid) the solve of a
// subdomain runs as two chains of about nl/2 line steps each, on the two CTAs
// of a cluster:
//   top (rank 0):    y_j = D_j (b_j - a_j y_{j-1})                     j = 0 .. mid-1
//                    u_mid = F (b_mid - a_mid y_{mid-1} - c_mid z_{mid+1})
//                    u_j = y_j - D_j (c_j u_{j+1})                      j = mid-1 .. 0
//   bottom (rank 1): z_j = E_j (b_j - c_j z_{j+1})                     j = nl-1 .. mid+1
//                    u_j = z_j - E_j (a_j u_{j-1})                      j = mid+1 .. nl-1
// (a_j couples line j to j-1, c_j to j+1; both are diagonal).  The halves meet
// once in each direction: the bottom stores z_{mid+1} (its line mid+1 of the
// output) and the top u_mid (line mid), each followed by one release arrive on
// the peer's barrier; the peer reads the line back from global memory after
// its acquire wait and applies the coupling itself.
// Each CTA holds all n rows of the block (NT = 2 M = 128 tiles for n <= 256,
// NT = 3 for n <= 384 with FP16 operands), so no data crosses between the
// CTAs during the line steps, and the chain of a level is about half as long
// as the one-ended solve's.  Every tile is one M = 128 MMA shape; the last
// tile's rows beyond the image (R = roundup16(n)) read the next stage or the
// ring's tail and land in accumulator lanes of no block row.
//
// Roles: warps 0 .. 4NT-1 epilogue (warp e: tile e/4, TMEM lanes 32*(e%4) ..);
// then kTwP bulk-copy producers and kTwP MMA issuers, one sub-ring of the
// operand ring per producer/issuer pair (stream positions q, q+kTwP, ...).
// An issuer takes each stage's tiles in turn and issues the four K = 16 MMAs
// of a 64-wide chunk back to back into one accumulator: measured, that keeps
// the tensor pipe near one M = 128, N = 16 MMA per ~47 cycles, where
// interleaving single MMAs over accumulators and tiles ran ~2.7x slower.
// Handshakes: full/empty per stage, acc_full per step, b_ready per step (B of
// the step written; B is single-buffered: the epilogue writes it only after
// every MMA of the previous step completed), x_in (the peer's middle line is
// in global memory; one phase).  Every wait is bounded; on expiry the CTA raises the device
// error word, each role leaves its loop, copies and MMAs are drained, the two
// CTAs drain the middle copies between them, and TMEM is freed.
// producer / issuer pairs: three for TF32 (288 KB of operand per line step),
// two for FP16 (half the bytes)
__host__ __device__ constexpr int tw_pairs(bool f16) { return f16 ? 2 : 3; }
// NT M = 128 tiles of block rows (n <= 128 NT), four epilogue warps each
__host__ __device__ constexpr int tw_threads(bool f16, int NT) { return 32 * (4 * NT + 2 * tw_pairs(f16)); }

// F16: operands in FP16 (kind::f16, K chunks of 64) with power-of-two
// scales: each factor line by 2^ascale[line] (set when the image is built),
// each right-hand-side column of B by a scale chosen every step from the
// column's largest value (a reduction over the CTA, which holds every row),
// so that both land in [2^13, 2^14); the FP32 accumulator is multiplied back
// by the inverse powers of two.  FP16 keeps TF32's 10-bit mantissa, so entries
// above ~2^-27 of their line's or column's largest carry the same rounding.
template <int PG, bool F16, int NT>
__global__ void __launch_bounds__(tw_threads(F16, NT)) solve_twist_kernel(
    const Task* __restrict__ tasks, const SubDesc* __restrict__ subs, int nrhs,
    const void* __restrict__ afac_v, const int64_t* __restrict__ afac_off, const int* __restrict__ ascale,
    const cplx<float>* __restrict__ Pv, const cplx<float>* __restrict__ inva, cplx<float>* buf,
    const cplx<float>* __restrict__ bsrc, int64_t rstride, int nstage, uint32_t ring_bytes, DevStatus ds) {
    constexpr int kN = 2 * PG;
    constexpr int kBChunkBytes = kN * 128;
    constexpr int kKc = F16 ? 64 : 32;  // K values per 128-byte row of a chunk
    constexpr int kTwP = tw_pairs(F16);
    constexpr int kTwEpi = 4 * NT;  // epilogue warps: tile e / 4, TMEM lanes 32 (e % 4) ..
    constexpr uint32_t kTwEpiThreads = 32 * kTwEpi;
    constexpr int kTwWarpProd = kTwEpi;
    constexpr int kTwWarpIss = kTwWarpProd + kTwP;
    const char* afac = reinterpret_cast<const char*>(afac_v);
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t rank = cluster_rank();  // 0: top half, 1: bottom half
    const uint32_t peer = rank ^ 1u;
    // cluster c = blockIdx.x / 2 is (task c / npanel, panel c % npanel): the
    // panels of a task are adjacent in launch order, so the CTAs that stream
    // the same factor lines are resident together and share them through L2
    const int npanel = (nrhs + PG - 1) / PG;
    const int cpair = blockIdx.x / 2, panel = cpair % npanel;
    const Task tk = tasks[cpair / npanel];
    const SubDesc& S = subs[tk.sub];
    const int n = S.nblk, nl = S.nlines, mid = nl / 2, nb = nl - 1 - mid;
    const int ntile = (n + 127) / 128;
    int nkc;
    const int64_t line_bytes = F16 ? umma_line_bytes16(n, &nkc) : umma_line_bytes(n, 1, &nkc);
    const int R = umma_rows(n, 1);
    const uint32_t stage_bytes = (uint32_t)R * 128;
    const int NS = nstage, NQ = NS / kTwP;
    const uint32_t b_bytes = (uint32_t)(nkc * kBChunkBytes);
    const int nsteps = rank == 0 ? 2 * mid + 1 : 2 * nb;
    // Whole-line ring: when one line of factors fits (chunk li in stage li, the
    // second tile's reads of the last chunk included), producer / issuer pair q
    // owns the contiguous chunks [q*cpp, q*cpp + cpp) and moves them with ONE
    // bulk copy per step (copies issued by one warp complete one after another,
    // so fewer, larger copies arrive sooner); otherwise the chunks are dealt
    // round-robin over kTwP sub-rings of NS/kTwP stages.
    const bool whole = (uint32_t)(nkc - 1) * stage_bytes + (uint32_t)(NT * kTileBytes) <= ring_bytes;
    const int cpp = (nkc + kTwP - 1) / kTwP;
    const int nq_act = whole ? (nkc + cpp - 1) / cpp : (nkc < kTwP ? nkc : kTwP);  // issuers with chunks
    // line of step s of this CTA
    auto line_of = [&](int st) -> int {
        if (rank == 0) return st < mid ? st : (st == mid ? mid : 2 * mid - st);
        return st < nb ? nl - 1 - st : mid + 1 + (st - nb);
    };

    // shared layout (1024-aligned): ring | B | per-line scalars | barriers | slots
    const uint32_t base = (su32(smem_raw) + 1023u) & ~1023u;
    unsigned char* gbase = smem_raw + (base - su32(smem_raw));
    const uint32_t stage0 = base;
    const uint32_t b0 = stage0 + ring_bytes;
    float* bl = reinterpret_cast<float*>(gbase + ring_bytes);
    // per-line scalars: 1/alpha at the nl+1 faces, then the FP16 line scales
    const uint32_t ls0 = b0 + b_bytes;
    cplx<float>* ia_s = reinterpret_cast<cplx<float>*>(gbase + (ls0 - base));
    int* as_s = reinterpret_cast<int*>(gbase + (ls0 - base) + (uint32_t)(nl + 1) * 8u);
    const uint32_t bars = (ls0 + (uint32_t)(nl + 1) * 8u + (uint32_t)nl * 4u + 7u) & ~7u;
    uint64_t* bars_g = reinterpret_cast<uint64_t*>(gbase + (bars - base));
    auto full = [&](int s) { return bars + 8u * s; };
    auto empty = [&](int s) { return bars + 8u * (NS + s); };
    const uint32_t acc_full = bars + 8u * (2 * NS);
    const uint32_t b_ready = bars + 8u * (2 * NS + 1);
    const uint32_t x_in = bars + 8u * (2 * NS + 2);
    const uint32_t drain = bars + 8u * (2 * NS + 3);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars_g + 2 * NS + 4);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    uint32_t* s_red = tmem_slot + 4;  // [2][kTwEpi][PG] column maxima (F16 scales), by step parity

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr uint32_t kCols = NT * kTwP * kN <= 32 ? 32 : NT * kTwP * kN <= 64 ? 64 :
                               NT * kTwP * kN <= 128 ? 128 : 256;  // tile t, issuer q: (t*kTwP + q)*kN
    static_assert(NT * kTwP * kN <= 256, "accumulators beyond 256 TMEM columns");

    if (tid == 0) {
        *abort_flag = 0;
        for (int s = 0; s < NS; ++s) {
            mb_init(full(s), 1);
            mb_init(empty(s), 1);
        }
        mb_init(acc_full, kTwP);
        mb_init(b_ready, kTwEpi);  // one arrival per epilogue warp
        mb_init(x_in, 1);
        mb_init(drain, kTwP);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (uint32_t i = tid; i < b_bytes / 4; i += blockDim.x) bl[i] = 0.f;
    {
        float* sg = reinterpret_cast<float*>(gbase);
        for (uint32_t i = tid; i < ring_bytes / 4; i += blockDim.x) sg[i] = 0.f;
    }
    if (warp == kTwWarpIss) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();  // the peer's barriers are initialised before its copy can land
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp >= kTwWarpProd && warp < kTwWarpProd + kTwP) {
        // ====================================================== producers
        const int pq = warp - kTwWarpProd;
        if (lane == 0 && whole) {
            const char* abase = afac + afac_off[tk.sub];
            const int c0q = pq * cpp, cnt = nkc - c0q < cpp ? nkc - c0q : cpp;
            int issued = 0;
            for (int step = 0; cnt > 0 && step < nsteps && !*abort_flag; ++step) {
                const int j = line_of(step);
                if (step > 0 && !mb_wait(empty(pq), (uint32_t)((step - 1) & 1), ds.polls)) {
                    atomicExch(ds.err, 2);
                    *abort_flag = 1;
                }
                if (*abort_flag) break;
                mb_expect_tx(full(pq), (uint32_t)cnt * stage_bytes);
                bulk_g2s(stage0 + (uint32_t)c0q * stage_bytes,
                         abase + (int64_t)j * line_bytes + (int64_t)c0q * stage_bytes, (uint32_t)cnt * stage_bytes,
                         full(pq));
                issued = step + 1;
            }
            // drain: the last copy lands (every earlier one was consumed)
            if (issued > 0) mb_wait(full(pq), (uint32_t)((issued - 1) & 1), kWait);
        } else if (lane == 0) {
            const char* abase = afac + afac_off[tk.sub];
            int k = 0;
            for (int step = 0; step < nsteps && !*abort_flag; ++step) {
                const int j = line_of(step);
                for (int li = pq; li < nkc; li += kTwP) {
                    const int s = pq * NQ + k % NQ;
                    if (k >= NQ && !mb_wait(empty(s), (uint32_t)(((k / NQ) - 1) & 1), ds.polls)) {
                        atomicExch(ds.err, 2);
                        *abort_flag = 1;
                    }
                    if (*abort_flag) break;
                    mb_expect_tx(full(s), stage_bytes);
                    bulk_g2s(stage0 + s * stage_bytes, abase + (int64_t)j * line_bytes + (int64_t)li * stage_bytes,
                             stage_bytes, full(s));
                    ++k;
                }
            }
            for (int kk = (k > NQ ? k - NQ : 0); kk < k; ++kk)
                mb_wait(full(pq * NQ + kk % NQ), (uint32_t)((kk / NQ) & 1), kWait);
        }
    } else if (warp >= kTwWarpIss && warp < kTwWarpIss + kTwP) {
        // ====================================================== MMA issuers
        const int q = warp - kTwWarpIss;
        if (lane == 0) {
            constexpr uint32_t idesc = F16 ? idesc_f16(128, kN) : idesc_tf32(128, kN);
            const uint64_t bdesc0 = desc_sw128(b0);
            int k = 0;
            for (int step = 0; step < nsteps && !*abort_flag; ++step) {
                if (!mb_wait(b_ready, (uint32_t)(step & 1), ds.polls)) {
                    atomicExch(ds.err, 2);
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                if (whole) {
                    const int c0q = q * cpp, cnt = nkc - c0q < cpp ? nkc - c0q : cpp;
                    if (cnt > 0) {
                        if (!mb_wait(full(q), (uint32_t)(step & 1), ds.polls)) {
                            atomicExch(ds.err, 2);
                            *abort_flag = 1;
                            break;
                        }
                        tc_fence_after();
                        for (int i = 0; i < cnt; ++i) {
                            const int li = c0q + i;
                            const uint64_t bdesc = bdesc0 + (uint64_t)(li * (kBChunkBytes >> 4));
                            for (int t = 0; t < ntile; ++t) {
                                const uint64_t adesc =
                                    desc_sw128(stage0 + (uint32_t)li * stage_bytes + (uint32_t)t * kTileBytes);
                                const uint32_t dacc = tmem + (uint32_t)((t * kTwP + q) * kN);
#pragma unroll
                                for (int kk = 0; kk < 4; ++kk) {
                                    if constexpr (F16)
                                        umma_f16(dacc, adesc + (uint64_t)(2 * kk), bdesc + (uint64_t)(2 * kk),
                                                 idesc, (i == 0 && kk == 0) ? 0u : 1u);
                                    else
                                        umma_tf32(dacc, adesc + (uint64_t)(2 * kk), bdesc + (uint64_t)(2 * kk),
                                                  idesc, (i == 0 && kk == 0) ? 0u : 1u);
                                }
                            }
                        }
                        umma_commit(empty(q));
                    }
                    umma_commit(acc_full);
                    continue;
                }
                bool first = true;
                for (int li = q; li < nkc; li += kTwP) {
                    const int s = q * NQ + k % NQ;
                    const uint32_t par = (uint32_t)((k / NQ) & 1);
                    ++k;
                    if (!mb_wait(full(s), par, ds.polls)) {
                        atomicExch(ds.err, 2);
                        *abort_flag = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t bdesc = bdesc0 + (uint64_t)(li * (kBChunkBytes >> 4));
                    for (int t = 0; t < ntile; ++t) {
                        const uint64_t adesc = desc_sw128(stage0 + s * stage_bytes + (uint32_t)t * kTileBytes);
                        const uint32_t dacc = tmem + (uint32_t)((t * kTwP + q) * kN);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            if constexpr (F16)
                                umma_f16(dacc, adesc + (uint64_t)(2 * kk), bdesc + (uint64_t)(2 * kk), idesc,
                                         (first && kk == 0) ? 0u : 1u);
                            else
                                umma_tf32(dacc, adesc + (uint64_t)(2 * kk), bdesc + (uint64_t)(2 * kk), idesc,
                                          (first && kk == 0) ? 0u : 1u);
                        }
                    }
                    first = false;
                    umma_commit(empty(s));
                }
                if (*abort_flag) break;
                umma_commit(acc_full);
            }
            umma_commit(drain);
            mb_wait(drain, 0u, kWait);
        }
    } else if (warp < kTwEpi) {
        // ====================================================== epilogue (warps 0 .. 4 NT - 1)
        const int t = warp / 4, quarter = warp % 4;
        const int p = t * 128 + quarter * 32 + lane;  // block row (TMEM lane quarter*32 + lane of tile t)
        const bool rv = p < n && t < ntile;
        const int n4 = (n + 3) & ~3;
        const bool wr = p < n4 && t < ntile;  // writes B rows 2p, 2p+1
        const cplx<float> pvp = rv ? Pv[S.coup_off + p] : mk<float>(0, 0);
        cplx<float>* V = buf + tk.buf_off;
        const int c0 = panel * PG;
        int ncol = nrhs - c0;
        if (ncol > PG) ncol = PG;
        const int k0 = 2 * p;
        const int kcb = k0 / kKc, kkb = k0 % kKc;
        // byte offset of B[row][k0] (k0 and k0+1 adjacent in one 16-byte unit)
        auto boff = [&](int row) -> uint32_t {
            if constexpr (F16)
                return (uint32_t)(kcb * kBChunkBytes + row * 128 + (((kkb / 8) ^ (row % 8)) * 16) + (kkb % 8) * 2);
            else
                return (uint32_t)(kcb * kBChunkBytes + row * 128 + (((kkb / 4) ^ (row % 8)) * 16) + (kkb % 4) * 4);
        };
        auto coup = [&](int face) -> cplx<float> { return rv ? pvp * ia_s[face] : mk<float>(0, 0); };
        int sbv[PG];  // F16: exponent of the scale of each column of the current B
#pragma unroll
        for (int c = 0; c < PG; ++c) sbv[c] = 0;
        const cplx<float>* Bsrc = bsrc + tk.buf_off;  // the local source b
        // line j of the source (b) or of this solve's own output (y, z)
        auto vload = [&](int j, bool src_b, cplx<float> (&dst)[PG]) {
            const cplx<float>* src = src_b ? Bsrc : V;
#pragma unroll
            for (int c = 0; c < PG; ++c)
                dst[c] = (rv && c < ncol && j >= 0) ? src[(int64_t)(c0 + c) * rstride + (int64_t)j * n + p]
                                                    : mk<float>(0, 0);
        };
        auto vstore = [&](int j, const cplx<float> (&v)[PG]) {
#pragma unroll
            for (int c = 0; c < PG; ++c)
                if (rv && c < ncol) V[(int64_t)(c0 + c) * rstride + (int64_t)j * n + p] = v[c];
        };
        // B of the next step: rows 2c (Re r, -Im r) and 2c+1 (Im r, Re r); the
        // epilogue's one barrier of the step (which also takes the uniform abort
        // decision over the step's waits, and for FP16 combines the column
        // maxima into the scale exponents) comes before any B write; then each
        // warp, its stores made visible to the tensor cores and its TMEM loads
        // ordered, arrives on b_ready.  False: some thread's wait failed.
        int ann = 0;
        auto announce = [&](const cplx<float> (&v)[PG], bool bad) -> bool {
            if constexpr (F16) {
                uint32_t* sr = s_red + (ann & 1) * (kTwEpi * PG);
#pragma unroll
                for (int c = 0; c < PG; ++c) {
                    const float m = rv ? fmaxf(fabsf(v[c].re), fabsf(v[c].im)) : 0.f;
                    const uint32_t wmx = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
                    if (lane == 0) sr[warp * PG + c] = wmx;
                }
                if (epi_any(bad, kTwEpiThreads)) return false;
                {
                    // lane c < PG combines column c over the epilogue warps; the
                    // exponents then reach every lane by shuffles
                    const int cl = lane < PG ? lane : 0;
                    uint32_t mx = 0;
#pragma unroll
                    for (int w = 0; w < kTwEpi; ++w) mx = max(mx, sr[w * PG + cl]);
                    int sc = 0;
                    if (mx != 0 && mx < 0x7F800000u) {
                        sc = 13 - ((int)((mx >> 23) & 0xFF) - 127);
                        sc = sc < -100 ? -100 : (sc > 100 ? 100 : sc);
                    }
#pragma unroll
                    for (int c = 0; c < PG; ++c) sbv[c] = __shfl_sync(0xffffffffu, sc, c);
                }
                if (wr) {
                    __half* bh = reinterpret_cast<__half*>(bl);
#pragma unroll
                    for (int c = 0; c < PG; ++c) {
                        const float s2 = pow2f(sbv[c]);
                        const float re = v[c].re * s2, im = v[c].im * s2;
                        *reinterpret_cast<__half2*>(bh + boff(2 * c) / 2) = __floats2half2_rn(re, -im);
                        *reinterpret_cast<__half2*>(bh + boff(2 * c + 1) / 2) = __floats2half2_rn(im, re);
                    }
                }
            } else {
                if (epi_any(bad, kTwEpiThreads)) return false;
                if (wr) {
#pragma unroll
                    for (int c = 0; c < PG; ++c) {
                        const float re = __uint_as_float(to_tf32(v[c].re)), im = __uint_as_float(to_tf32(v[c].im));
                        const float nim = __uint_as_float(to_tf32(-v[c].im));
                        *reinterpret_cast<float2*>(bl + boff(2 * c) / 4) = make_float2(re, nim);
                        *reinterpret_cast<float2*>(bl + boff(2 * c + 1) / 4) = make_float2(im, re);
                    }
                }
            }
            ++ann;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b_ready) : "memory");
            return true;
        };
        // middle line to the peer: this CTA's rows of line lm stored to the
        // output (made visible at cluster scope), then one release arrive on
        // the peer's x_in
        auto send_middle = [&](int lm, const cplx<float> (&v)[PG]) {
            vstore(lm, v);
            fence_acq_rel_cluster();
            epi_sync(kTwEpiThreads);
            if (tid == 0) mb_arrive_remote(map_peer(x_in, peer));
        };
        // the peer's line lm times the coupling cf (every epilogue thread waits;
        // uniform outcome)
        auto recv_middle = [&](int lm, cplx<float> cf, cplx<float> (&dst)[PG]) -> bool {
            const bool got = mb_wait_cluster(x_in, 0u, ds.polls);
            if (epi_any(!got, kTwEpiThreads)) return false;
#pragma unroll
            for (int c = 0; c < PG; ++c)
                dst[c] = (rv && c < ncol) ? cf * V[(int64_t)(c0 + c) * rstride + (int64_t)lm * n + p]
                                          : mk<float>(0, 0);
            return true;
        };
        // operand kept from memory for the epilogue of step st: top: b_{st+1}
        // (forward), y_j (backward); bottom: b_{j-1} (forward), z_j (backward)
        auto pre_line = [&](int st) -> int {
            if (st >= nsteps) return -1;
            if (rank == 0) return st < mid ? st + 1 : (st == mid ? -1 : 2 * mid - st);
            if (st < nb) return (nl - 2 - st > mid) ? nl - 2 - st : -1;
            return mid + 1 + (st - nb);
        };
        // the forward steps' operand is the source b, the backward steps' their y / z
        auto pre_is_b = [&](int st) -> bool { return rank == 0 ? st < mid : st < nb; };
        cplx<float> pre[PG], pre_next[PG], outv[PG], nbv[PG], xv[PG];
        // this subdomain's per-line scalars into shared memory (off the step chain)
        for (int f = tid; f <= nl; f += kTwEpiThreads) ia_s[f] = inva[S.inva_off + f];
        if constexpr (F16)
            for (int f = tid; f < nl; f += kTwEpiThreads) as_s[f] = ascale[S.inva_off + f];
        // first B: b_0 (top) or b_{nl-1} (bottom)
        vload(rank == 0 ? 0 : nl - 1, true, nbv);
        vload(pre_line(0), pre_is_b(0), pre);
        epi_sync(kTwEpiThreads);
        bool ok = announce(nbv, false);
        for (int step = 0; ok && step < nsteps; ++step) {
            const int j = line_of(step);
            vload(pre_line(step + 1), pre_is_b(step + 1), pre_next);
            // a failed wait is acted on at the step's barrier (uniformly); the
            // TMEM loads below stay within this CTA's allocation either way
            const bool bad = *abort_flag || !mb_wait(acc_full, (uint32_t)(step & 1), ds.polls);
            tc_fence_after();
            float acc[kN];
#pragma unroll
            for (int e = 0; e < kN; ++e) acc[e] = 0.f;
            {
                uint32_t part[kTwP][kN / 16][16];
#pragma unroll
                for (int q = 0; q < kTwP; ++q)
#pragma unroll
                    for (int h = 0; h < kN / 16; ++h)
                        if (q < nq_act)
                            tmem_ld16_async(tmem + ((uint32_t)(quarter * 32) << 16) +
                                                (uint32_t)(((t < ntile ? t : 0) * kTwP + q) * kN + 16 * h),
                                            part[q][h]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int q = 0; q < kTwP; ++q)
#pragma unroll
                    for (int h = 0; h < kN / 16; ++h) {
                        if (q >= nq_act) continue;
                        tmem_pin16(part[q][h]);
#pragma unroll
                        for (int e = 0; e < 16; ++e) acc[16 * h + e] += __uint_as_float(part[q][h][e]);
                    }
            }
            cplx<float> y[PG];
            if constexpr (F16) {
                const int sa = as_s[j];
#pragma unroll
                for (int c = 0; c < PG; ++c) {
                    const float us = pow2f(-(sa + sbv[c]));
                    y[c] = mk<float>(acc[2 * c] * us, acc[2 * c + 1] * us);
                }
            } else {
#pragma unroll
                for (int c = 0; c < PG; ++c) y[c] = mk<float>(acc[2 * c], acc[2 * c + 1]);
            }
            bool last = step + 1 >= nsteps;
            bool stored = false;  // outv already in the output (a middle line)
            if (rank == 0) {
                if (step < mid) {  // y_j; next: b_{j+1} - a_{j+1} y_j (minus the bottom's c_mid z_{mid+1} at mid)
                    const cplx<float> a = coup(j + 1);
#pragma unroll
                    for (int c = 0; c < PG; ++c) {
                        outv[c] = y[c];
                        nbv[c] = rv ? pre[c] - a * y[c] : mk<float>(0, 0);
                    }
                    if (step + 1 == mid) {  // the bottom's c_mid z_{mid+1}
                        if (!recv_middle(mid + 1, coup(mid + 1), xv)) { ok = false; break; }
#pragma unroll
                        for (int c = 0; c < PG; ++c) nbv[c] = rv ? nbv[c] - xv[c] : mk<float>(0, 0);
                    }
                } else if (step == mid) {  // u_mid, to the bottom; next: c_{mid-1} u_mid
                    const cplx<float> cc = coup(mid);
#pragma unroll
                    for (int c = 0; c < PG; ++c) {
                        outv[c] = y[c];
                        nbv[c] = rv ? cc * y[c] : mk<float>(0, 0);
                    }
                    if (nb > 0) {
                        send_middle(mid, outv);
                        stored = true;
                    }
                } else {  // u_j = y_j - D_j (c_j u_{j+1}); next: c_{j-1} u_j
                    const cplx<float> cc = coup(j);
#pragma unroll
                    for (int c = 0; c < PG; ++c) {
                        outv[c] = pre[c] - y[c];
                        nbv[c] = rv ? cc * outv[c] : mk<float>(0, 0);
                    }
                }
            } else {
                if (step < nb) {  // z_j; next: b_{j-1} - c_{j-1} z_j, or at mid+1: the top's a_{mid+1} u_mid
                    const cplx<float> cc = coup(j);
#pragma unroll
                    for (int c = 0; c < PG; ++c) {
                        outv[c] = y[c];
                        nbv[c] = rv ? pre[c] - cc * y[c] : mk<float>(0, 0);
                    }
                    if (step + 1 == nb) {  // z_{mid+1} to the top; back: a_{mid+1} u_mid
                        send_middle(mid + 1, outv);
                        stored = true;
                        if (!recv_middle(mid, coup(mid + 1), xv)) { ok = false; break; }
#pragma unroll
                        for (int c = 0; c < PG; ++c) {
                            nbv[c] = rv ? xv[c] : mk<float>(0, 0);
                            pre_next[c] = y[c];  // z_{mid+1}, the first backward step's y
                        }
                    }
                } else {  // u_j = z_j - E_j (a_j u_{j-1}); next: a_{j+1} u_j
                    const cplx<float> a = coup(j + 1);
#pragma unroll
                    for (int c = 0; c < PG; ++c) {
                        outv[c] = pre[c] - y[c];
                        nbv[c] = rv ? a * outv[c] : mk<float>(0, 0);
                    }
                }
            }
            if (last ? epi_any(bad, kTwEpiThreads) : !announce(nbv, bad)) {
                ok = false;
                break;
            }
            if (!stored) vstore(j, outv);
#pragma unroll
            for (int c = 0; c < PG; ++c) pre[c] = pre_next[c];
        }
        if (!ok) {
            atomicExch(ds.err, 2);
            *abort_flag = 1;
        }
    }
    tc_fence_before();
    __syncthreads();
    // neither CTA leaves while the peer's arrive on its x_in may be in flight
    cluster_sync();
    tc_fence_after();
    if (warp == kTwWarpIss)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

// Shared-memory plan of a twisted launch: ns stages (kTwP sub-rings of at
// least 2) of R*128 bytes, the last one at least NT tiles long (the last
// tile's MMA reads 128 rows), B, the per-line scalars, barriers, slots and the
// column-maximum scratch, alignment; 0 if it does not fit.
static size_t twist_smem_plan(int PG, bool f16, int NT, int nblk_max, int nlines_max, int* ns_out,
                              uint32_t* ring_out) {
    const int kTwP = tw_pairs(f16);
    int nkc = 0;
    if (f16)
        umma_line_bytes16(nblk_max, &nkc);
    else
        umma_line_bytes(nblk_max, 1, &nkc);
    const size_t sb = (size_t)umma_rows(nblk_max, 1) * 128;
    const size_t tail = (size_t)NT * kTileBytes;  // the last tile's MMA reads 128 rows from +16 (NT-1) KB
    const size_t lines = (size_t)(nlines_max + 1) * 8 + (size_t)nlines_max * 4;
    const size_t fixed = (size_t)nkc * 2 * PG * 128 + lines + 1024 + 1024;
    const size_t budget = 227 * 1024;
    if (fixed + (2 * kTwP - 1) * sb + tail > budget) return 0;
    int ns = (int)((budget - fixed - tail) / sb) + 1;
    // (2 ns + 4) barriers, 4 slots and the 2 x 4NT x PG column-maximum scratch
    // within the 1 KB reserve (8 of it for the barriers' alignment)
    const int ns_cap = ((1024 - 8 - 16 - 2 * 4 * NT * PG * 4) / 8 - 4) / 2;
    if (ns > ns_cap) ns = ns_cap;
    ns -= ns % kTwP;
    if (ns < 2 * kTwP) return 0;
    *ns_out = ns;
    *ring_out = (uint32_t)((ns - 1) * sb + tail);
    return *ring_out + fixed;
}

// Tiles of the twisted launch: two up to 256 block rows, three up to 384
// (FP16 only: the TF32 ring of a 384-row block does not fit next to B).
static int twist_tiles(int nblk_max) { return nblk_max <= 256 ? 2 : 3; }

bool twist_supported(int nblk_max, int nlines_min, int nlines_max, bool f16) {
    int ns;
    uint32_t ring;
    return nblk_max <= (f16 ? 384 : 256) && nlines_min >= 4 &&
           twist_smem_plan(8, f16, twist_tiles(nblk_max), nblk_max, nlines_max, &ns, &ring) != 0;
}

int64_t twist_f16_factor_bytes(const SubDesc& S) { return umma_line_bytes16(S.nblk, nullptr) * S.nlines; }

void launch_line_scales(const SubDesc* subs_d, int nsub, int max_lines, const float* fac, const float* fac2,
                        int* ascale, cudaStream_t st) {
    line_scale_kernel<<<dim3(nsub, max_lines), 256, 0, st>>>(subs_d, fac, fac2, ascale);
}

void launch_repack_f16(const SubDesc* subs_d, const std::vector<SubDesc>& subs_h, const float* fac,
                       const float* fac2, const int* ascale, const int64_t* dst_off_d, void* dst,
                       cudaStream_t st) {
    for (size_t s = 0; s < subs_h.size(); ++s) {
        const int64_t halves = umma_line_bytes16(subs_h[s].nblk, nullptr) / 2 * subs_h[s].nlines;
        repack_f16_kernel<<<(unsigned)((halves + 255) / 256), 256, 0, st>>>(
            subs_d, fac, fac2, ascale, dst_off_d, static_cast<__half*>(dst), (int)s);
    }
}

template <bool F16, int NT>
static void launch_twist_t(const Task* tasks, int ntask, const SubDesc* subs, int nblk_max, int nlines_max, int nrhs,
                           const void* afac, const int64_t* afac_off, const int* ascale, const cplx<float>* Pv,
                           const cplx<float>* inva, cplx<float>* buf, const cplx<float>* bsrc, int64_t rstride,
                           DevStatus ds, cudaStream_t st) {
    constexpr int PG = 8;
    int ns = 0;
    uint32_t ring = 0;
    const size_t smem = twist_smem_plan(PG, F16, NT, nblk_max, nlines_max, &ns, &ring);
    cudaFuncSetAttribute(solve_twist_kernel<PG, F16, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ntask * 2 * ((nrhs + PG - 1) / PG), 1, 1);
    cfg.blockDim = dim3(tw_threads(F16, NT), 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, solve_twist_kernel<PG, F16, NT>, tasks, subs, nrhs, afac, afac_off, ascale, Pv, inva,
                       buf, bsrc, rstride, ns, ring, ds);
}

void launch_solve_twist(const Task* tasks, int ntask, const SubDesc* subs, int nblk_max, int nlines_max, int nrhs,
                        const void* afac, const int64_t* afac_off, const int* ascale, bool f16,
                        const cplx<float>* Pv, const cplx<float>* inva, cplx<float>* buf,
                        const cplx<float>* bsrc, int64_t rstride, DevStatus ds, cudaStream_t st) {
    if (ntask == 0) return;
    if (f16 && twist_tiles(nblk_max) == 3)
        launch_twist_t<true, 3>(tasks, ntask, subs, nblk_max, nlines_max, nrhs, afac, afac_off, ascale, Pv, inva, buf,
                                bsrc, rstride, ds, st);
    else if (f16)
        launch_twist_t<true, 2>(tasks, ntask, subs, nblk_max, nlines_max, nrhs, afac, afac_off, ascale, Pv, inva, buf,
                                bsrc, rstride, ds, st);
    else
        launch_twist_t<false, 2>(tasks, ntask, subs, nblk_max, nlines_max, nrhs, afac, afac_off, ascale, Pv, inva, buf,
                                 bsrc, rstride, ds, st);
}

}  // namespace helm
