// scan_tc.cu -- distance tiles in the tensor-core Gram form (tcgen05, sm_103a).
//
// For globally normalised subsequences x, y of length n with means mu_x,
// mu_y and centred parts x' = x - mu_x, y' = y - mu_y (sum x' = sum y' = 0):
//     ||x - y||^2 = c_x + c_y + n (mu_x - mu_y)^2 - 2 <x', y'>,
// c = ||x'||^2 (Eq. 1 squared, rewritten so that no large uncentred norms
// cancel).  <x', y'> for a 128-row x 256-column tile is one tcgen05 UMMA
// chain (M=128, N=256, K=16 per instruction, FP16 or BF16 operands staged by
// 128-byte-swizzled TMA loads, FP32 accumulators in tensor memory); the
// epilogue warps read the accumulators back with tcgen05.ld and finish the
// distance, the exclusion zone |i - j| < n and the running row minimum.
//
// Every row carries a rigorous bound F_i(D) on |D - d^2| for a computed
// distance D (operand rounding, FP32 accumulation, FP32 epilogue), so the
// search can abandon a row only when D + F_i(D) < best-so-far (a proven
// lower bound), and every row that the bound cannot rule out is rescored
// exactly in FP64 (rescore.cu).
//
// Roles (192 threads, one CTA per SM, persistent):
//   warp 0  lane 0 : TMA producer (A tile resident per item, B tiles through a ring)
//   warp 1         : TMEM allocation (512 columns = two 128x256 FP32 buffers);
//                    lane 0 issues the UMMAs and commits them to mbarriers
//   warps 2-5      : epilogue, one tile row per thread (TMEM lane = row)
// All mbarrier waits are bounded with %globaltimer; on expiry the CTA records
// DD_ETIMEOUT in the control block, drains and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dd_internal.cuh"

namespace dd {
namespace {

constexpr int TBM = 128;
constexpr int TBN = 256;
constexpr int TKA = 64;  // 16-bit elements per 128-byte swizzle atom
constexpr int kTcThreads = 192;
constexpr int kABytesPerAtom = TBM * 128;  // 16 KB
constexpr int kBBytesPerAtom = TBN * 128;  // 32 KB
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s

struct TcHdr {
    unsigned long long a_full;
    unsigned long long b_full[8];
    unsigned long long b_empty[8];
    unsigned long long acc_full[2];
    unsigned long long acc_empty[2];
    uint32_t tmem_base;
    int item;
    int abort;
    int pad;
    float4 col[2][TBN];
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned long long* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase of parity `parity`; false on timeout or abort.
__device__ bool mbar_wait(unsigned long long* bar, uint32_t parity, volatile int* abort) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255u) == 0u) {
            if (*abort) return false;
            if (globaltimer() - t0 > kWaitNs) return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, unsigned long long* bar, int x,
                                            int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::
            "r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void umma_commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;              // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;    // stride byte offset
    d |= (uint64_t)1u << 46;              // descriptor version for tcgen05
    d |= (uint64_t)2u << 61;              // 128-byte swizzle
    return d;
}

__device__ __forceinline__ float bound_F(float D, float alpha, float gam, float q2, float beta) {
    return alpha + beta * D + gam * sqrtf(fmaxf(D, 0.f) + q2);
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_scan_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, TcArgs a) {
    extern __shared__ unsigned char smraw[];
    // 1024-byte aligned operand area (128-byte swizzle atoms)
    const uint32_t base_u32 = smem_u32(smraw);
    const uint32_t pad = (1024u - (base_u32 & 1023u)) & 1023u;
    unsigned char* sbase = smraw + pad;
    unsigned char* sA = sbase;
    unsigned char* sB = sbase + a.nka * kABytesPerAtom;
    TcHdr& h = *reinterpret_cast<TcHdr*>(sB + a.stages * kBBytesPerAtom);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const Ctrl* ctrl = a.ctrl;
    if (ctrl->nonfinite || ctrl->degenerate) return;
    const int cnt = *a.rows.cnt_dev;
    const int off = a.rows.off_dev ? *a.rows.off_dev : 0;
    const int RT = (cnt + TBM - 1) / TBM;
    if (RT <= 0) return;
    long long items;
    int nseg0 = 1;
    if (a.mode == 2) {
        const int smax = *a.smax;
        if (smax <= 0) return;
        items = (long long)RT * smax;
    } else {
        nseg0 = (a.N + a.seg_cols - 1) / a.seg_cols;
        items = (long long)RT * nseg0;
    }

    if (tid == 0) {
        mbar_init(&h.a_full, 1);
        for (int s = 0; s < a.stages; s++) {
            mbar_init(&h.b_full[s], 1);
            mbar_init(&h.b_empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&h.acc_full[b], 1);
            mbar_init(&h.acc_empty[b], 128);
        }
        h.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(&h.tmem_base, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = h.tmem_base;
    volatile int* abort = &h.abort;

    // pipeline state (identical sequences in the producer and MMA roles)
    uint32_t a_phase = 0;
    int bstage = 0;
    uint32_t bphase = 0;
    uint32_t acc_phase[2] = {0u, 0u};
    const float neg2s = (float)(-2.0 / (a.stats[3] * a.stats[3]));  // s is a power of two: exact
    const int n = a.n;
    unsigned long long pairs = 0;

    for (;;) {
        __syncthreads();
        if (tid == 0) h.item = atomicAdd(&a.ctrl->work[a.work_slot], 1);
        __syncthreads();
        const int item = h.item;
        if (item >= items || *abort) break;
        int rt, pa, pb, dir;
        if (a.mode == 2) {
            const int s_rank = item / RT;
            rt = item % RT;
            const int4 r = a.ranges[rt];
            if (s_rank >= r.w) continue;
            const int side = s_rank & 1, idx = s_rank >> 1;
            if (side == 0) {
                pa = r.z + idx * a.seg_cols;
                pb = min(pa + a.seg_cols, r.y);
                dir = 1;
            } else {
                pb = r.z - idx * a.seg_cols;
                pa = max(pb - a.seg_cols, r.x);
                dir = -1;
            }
        } else {
            rt = item / nseg0;
            const int sg = item % nseg0;
            pa = sg * a.seg_cols;
            pb = min(pa + a.seg_cols, a.N);
            dir = 1;
        }
        if (pa >= pb) continue;
        const int nct = (pb - pa + TBN - 1) / TBN;

        // rows of the tile (epilogue threads own one row each)
        const bool epi = warp >= 2;
        const int r_in = epi ? ((warp & 3) * 32 + lane) : 0;
        int ri = -1;
        float rmu = 0.f, rc = 0.f, al = 0.f, ga = 0.f, q2 = 0.f, Drun = INFINITY, Dlast = INFINITY;
        if (epi) {
            const int r = rt * TBM + r_in;
            ri = r < cnt ? a.rows.base[off + r] : -1;
            if (ri >= 0) {
                rmu = a.rowmu[ri];
                rc = a.rowc[ri];
                al = a.alpha[ri];
                ga = a.gam[ri];
                q2 = a.q2[ri];
                Drun = __uint_as_float(a.rmin[ri]);
                Dlast = Drun;
            }
        }
        bool alive = true;
        if (a.abandon) {
            bool al_me = false;
            if (ri >= 0) {
                const float g = __uint_as_float(*((volatile const unsigned*)(a.rmin + ri)));
                const float D = fminf(Drun, g);
                const float bsf = __uint_as_float(*((volatile const unsigned*)&ctrl->bsf));
                al_me = !(D + bound_F(D, al, ga, q2, a.beta) < bsf);
            }
            alive = __syncthreads_or(al_me) != 0;
        }
        if (!alive) continue;

        if (warp == 0) {
            if (lane == 0) {
                // A tile: the 128 rows of the list tile, all k atoms
                const int arow = a.a_row0 + rt * TBM + (a.a_direct ? off : 0);
                mbar_expect_tx(&h.a_full, (uint32_t)(a.nka * kABytesPerAtom));
                for (int ka = 0; ka < a.nka; ka++) tma_load_2d(sA + ka * kABytesPerAtom, &mapA, &h.a_full, ka * TKA, arow);
                for (int ct = 0; ct < nct; ct++) {
                    const int p0 = dir > 0 ? pa + ct * TBN : pb - (ct + 1) * TBN;
                    for (int ka = 0; ka < a.nka; ka++) {
                        if (!mbar_wait(&h.b_empty[bstage], bphase ^ 1u, abort)) {
                            atomicExch(&a.ctrl->err, DD_ETIMEOUT);
                            *abort = 1;
                            break;
                        }
                        mbar_expect_tx(&h.b_full[bstage], (uint32_t)kBBytesPerAtom);
                        tma_load_2d(sB + bstage * kBBytesPerAtom, &mapB, &h.b_full[bstage], ka * TKA, p0);
                        if (++bstage == a.stages) {
                            bstage = 0;
                            bphase ^= 1u;
                        }
                    }
                    if (*abort) break;
                }
            }
        } else if (warp == 1) {
            if (lane == 0) {
                bool ok = mbar_wait(&h.a_full, a_phase, abort);
                a_phase ^= 1u;
                for (int ct = 0; ct < nct && ok; ct++) {
                    const int buf = ct & 1;
                    if (!mbar_wait(&h.acc_empty[buf], acc_phase[buf] ^ 1u, abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dt = tbase + (uint32_t)(buf * TBN);
                    for (int ka = 0; ka < a.nka; ka++) {
                        if (!mbar_wait(&h.b_full[bstage], bphase, abort)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t ad = sw128_desc(smem_u32(sA + ka * kABytesPerAtom));
                        const uint64_t bd = sw128_desc(smem_u32(sB + bstage * kBBytesPerAtom));
#pragma unroll
                        for (int kk = 0; kk < TKA / 16; kk++)
                            umma_f16(dt, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), a.idesc,
                                     (ka | kk) != 0 ? 1u : 0u);
                        umma_commit(&h.b_empty[bstage]);
                        if (++bstage == a.stages) {
                            bstage = 0;
                            bphase ^= 1u;
                        }
                    }
                    if (!ok) break;
                    umma_commit(&h.acc_full[buf]);
                    acc_phase[buf] ^= 1u;
                }
                if (!ok) {
                    atomicExch(&a.ctrl->err, DD_ETIMEOUT);
                    *abort = 1;
                }
            }
            __syncwarp();
        } else {
            // epilogue
            const int e = tid - 64;
            const int q = warp & 3;
            for (int ct = 0; ct < nct; ct++) {
                const int buf = ct & 1;
                const int p0 = dir > 0 ? pa + ct * TBN : pb - (ct + 1) * TBN;
#pragma unroll
                for (int k2 = 0; k2 < 2; k2++) {
                    const int c = e + k2 * 128;
                    const int p = p0 + c;
                    float4 cd;
                    if (p >= pa && p < pb) {
                        cd.x = a.colmu[p];
                        cd.y = a.colc[p];
                        cd.z = __int_as_float(a.sig[p]);
                    } else {
                        cd.x = 0.f;
                        cd.y = INFINITY;
                        cd.z = __int_as_float(-(1 << 30));
                    }
                    cd.w = 0.f;
                    h.col[buf][c] = cd;
                }
                // every epilogue thread reaches this barrier on every tile, abort or not
                asm volatile("bar.sync 1, 128;" ::: "memory");
                bool ok = !*abort && mbar_wait(&h.acc_full[buf], acc_phase[buf], abort);
                acc_phase[buf] ^= 1u;
                ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-wide
                if (!ok) {
                    atomicExch(&a.ctrl->err, DD_ETIMEOUT);
                    *abort = 1;
                    continue;
                }
                tc_fence_after();
                float m = INFINITY;
                const uint32_t taddr = tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * TBN);
#pragma unroll 1
                for (int ch = 0; ch < TBN / 32; ch++) {
                    uint32_t v[32];
                    tmem_ld32(taddr + (uint32_t)(ch * 32), v);
                    tmem_ld_wait();
#pragma unroll
                    for (int x = 0; x < 32; x++) {
                        const float4 cd = h.col[buf][ch * 32 + x];
                        const float dm = rmu - cd.x;
                        float t = fmaf(dm, dm, cd.y);
                        t = fmaf(neg2s, __uint_as_float(v[x]), t);
                        const int j = __float_as_int(cd.z);
                        const bool okc = (unsigned)(j - ri + n - 1) >= (unsigned)(2 * n - 1);
                        m = okc ? fminf(m, t) : m;
                    }
                }
                tc_fence_before();
                mbar_arrive(&h.acc_empty[buf]);
                const float D = fmaxf(m + rc, 0.f);
                Drun = fminf(Drun, D);
            }
            if (ri >= 0 && Drun < Dlast) atomicMin(a.rmin + ri, __float_as_uint(Drun));
            if (e == 0) {
                const int nvr = min(TBM, cnt - rt * TBM);
                pairs += (unsigned long long)nvr * (unsigned long long)(pb - pa);
            }
        }
    }
    __syncthreads();
    if (*abort && tid == 0) {
        // an expired wait: give copies already issued by this CTA time to land
        const unsigned long long t0 = globaltimer();
        while (globaltimer() - t0 < 200000ull) {
        }
    }
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tbase, 512);
    if (tid == 64 && pairs) atomicAdd(&a.ctrl->pairs, pairs);
}

// ---------------------------------------------------------------------------
// Preparation for the Gram form.

// Per row (orig order) and per column (mean-bucketed order): sqrt(n) mu_i,
// c_i (FP32), sqrt(c_i) rounded up; maxima over all rows.
__global__ void __launch_bounds__(256) k_tc_rowconst(const double* __restrict__ mu_w, const double* __restrict__ c_w,
                                                     const int32_t* __restrict__ sigpos, int64_t N, int n,
                                                     float* __restrict__ colmu, float* __restrict__ colc,
                                                     float* __restrict__ rowmu, float* __restrict__ rowc,
                                                     float* __restrict__ rowsc, Ctrl* ctrl) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float sc = 0.f, cc = 0.f, am = 0.f;
    if (i < N) {
        const double sn = sqrt((double)n);
        const float mu = (float)(sn * mu_w[i]);
        const float c = (float)c_w[i];
        sc = __double2float_ru(sqrt(c_w[i]));
        cc = __double2float_ru(c_w[i]);
        am = fabsf(mu);
        const int p = sigpos[i];
        colmu[p] = mu;
        colc[p] = c;
        rowmu[i] = mu;
        rowc[i] = c;
        rowsc[i] = sc;
    }
    // non-negative floats order like their bit patterns
    const unsigned bsc = __reduce_max_sync(0xffffffffu, __float_as_uint(sc));
    const unsigned bcc = __reduce_max_sync(0xffffffffu, __float_as_uint(cc));
    const unsigned bam = __reduce_max_sync(0xffffffffu, __float_as_uint(am));
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&ctrl->tc_scmax, bsc);
        atomicMax(&ctrl->tc_cmax, bcc);
        atomicMax(&ctrl->tc_mumax, bam);
    }
}

// Per-row error bound F_i(D) = alpha_i + beta D + gam_i sqrt(D + q2_i) on
// |D - d^2| for a distance D computed by the Gram tiles (safety factor 2):
//   operands rounded to u_in (FP16 2^-11, BF16 2^-8), products exact in FP32,
//   accumulation of n terms with unit 2^-23 (directed rounding allowed):
//     |g~ - g| <= ((2 u_in + u_in^2) + gamma_n (1 + u_in)^2) sum|x'y'|,
//     sum|x'y'| <= sqrt(c_i) sqrt(c_j) <= sc_i sc_max = Q_i;
//   subnormal operands add <= 2^-25 / s per element (scale s);
//   FP32 rounding of c~, sqrt(n) mu~, the epilogue FMAs and the final sum is
//   bounded through dm^2 <= D + 2 Q_i and |dm| <= sqrt(D + 2 Q_i).
__global__ void __launch_bounds__(256) k_tc_rowbound(const float* __restrict__ rowsc, const float* __restrict__ rowc,
                                                     const float* __restrict__ rowmu, int64_t N, int n, double u_in,
                                                     const double* stats, const double* P2end, const Ctrl* ctrl,
                                                     float* __restrict__ alpha, float* __restrict__ gam,
                                                     float* __restrict__ q2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double u32 = 5.9604644775390625e-08;  // 2^-24
    const double uacc = 2.384185791015625e-07; // 2^-22: allows truncating accumulation
    const double scmax = (double)__uint_as_float(ctrl->tc_scmax);
    const double cmax = (double)__uint_as_float(ctrl->tc_cmax);
    const double mumax = (double)__uint_as_float(ctrl->tc_mumax);
    const double s = stats[3];
    const double gn = n * uacc / (1.0 - n * uacc);
    const double Kg = 2.0 * ((2.0 * u_in + u_in * u_in) + gn * (1.0 + u_in) * (1.0 + u_in));
    const double sci = (double)rowsc[i];
    const double Q = sci * scmax;
    const double ci = (double)rowc[i];
    const double eta = 2.0 * (2.9802322387695312e-08 / s * sqrt((double)n) * (sci + scmax) +
                              (double)n * 8.881784197001252e-16 / (s * s));
    const double ec = 512.0 * 1.1102230246251565e-16 * (1.0 + *P2end);
    const double A0 = Kg * Q + eta + 2.0 * u32 * (ci + cmax) + 2.0 * ec + 8.0 * u32 * Q + 2.0 * u32 * (ci + cmax);
    const double G0 = 2.0 * u32 * (fabs((double)rowmu[i]) + mumax);
    alpha[i] = __double2float_ru(2.0 * A0);
    gam[i] = __double2float_ru(2.0 * G0);
    q2[i] = __double2float_ru(2.0 * Q);
}

__device__ __forceinline__ __half to16(double x, __half*) { return __double2half(x); }
__device__ __forceinline__ __nv_bfloat16 to16(double x, __nv_bfloat16*) { return __double2bfloat16(x); }

// Centred rows in the mean-bucketed order: S[p][k] = s (t^_{i+k} - mu_i),
// i = sig[p], rounded once to FP16 / BF16; zero for k in [n, kpad).
template <typename T16>
__global__ void __launch_bounds__(256) k_build_S(const double* __restrict__ t64, const double* __restrict__ mu_w,
                                                 const int32_t* __restrict__ sig, int64_t N, int n, int kpad,
                                                 const double* stats, T16* __restrict__ S) {
    const int per_row = kpad / 8;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t p = g / per_row;
    const int k0 = (int)(g % per_row) * 8;
    if (p >= N) return;
    const double s = stats[3];
    const int i = sig[p];
    const double mu = mu_w[i];
    T16 v[8];
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const int k = k0 + q;
        const double x = k < n ? (t64[i + k] - mu) * s : 0.0;
        v[q] = to16(x, (T16*)nullptr);
    }
    *reinterpret_cast<uint4*>(S + p * kpad + k0) = *reinterpret_cast<uint4*>(v);
}

// Operand scale: a power of two that puts max |x'| <= 2 max|t^| near 2^14 (FP16).
__global__ void k_tc_scale(double* stats, int is_bf16) {
    if (threadIdx.x != 0) return;
    double s = 1.0;
    if (!is_bf16) {
        const double mx = 2.0 * stats[2];
        if (mx > 0.0) {
            int e = (int)floor(log2(16384.0 / mx));
            if (e > 24) e = 24;
            if (e < -24) e = -24;
            s = ldexp(1.0, e);
        }
    }
    stats[3] = s;
}

// Packs the operand rows of a list (in list order) for TMA.
__global__ void __launch_bounds__(256) k_gather_rows(ListRef L, const int32_t* __restrict__ sigpos,
                                                     const uint4* __restrict__ S, int kpad, uint4* __restrict__ P) {
    const int cnt = *L.cnt_dev;
    const int off = L.off_dev ? *L.off_dev : 0;
    const int per_row = kpad / 8;  // uint4 per row
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r = g / per_row;
    const int c = (int)(g % per_row);
    if (r >= cnt) return;
    const int i = L.base[off + r];
    P[r * per_row + c] = S[(int64_t)sigpos[i] * per_row + c];
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        fn = reinterpret_cast<EncodeTiledFn>(ptr);
    }
    return fn;
}

bool make_map(CUtensorMap* map, void* base, int64_t rows, int kpad, int box_rows, bool bf16) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
    cuuint32_t box[2] = {(cuuint32_t)TKA, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, base, dims,
                    strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

size_t tc_smem_bytes(int kpad) {
    const int nka = kpad / TKA;
    const int stages = tc_stages(kpad);
    return 1024 + (size_t)nka * kABytesPerAtom + (size_t)stages * kBBytesPerAtom + sizeof(TcHdr);
}

int tc_stages(int kpad) {
    const int nka = kpad / TKA;
    const int budget = 200 * 1024 - nka * kABytesPerAtom;
    int st = budget / kBBytesPerAtom;
    if (st > 4) st = 4;
    return st;
}

bool tc_supported(int n) {
    const int kpad = (n + TKA - 1) / TKA * TKA;
    return kpad <= 512 && tc_stages(kpad) >= 2;
}

cudaError_t tc_make_maps(dd_plan_s* p) {
    const bool bf16 = p->opt.precision == DD_TC_BF16;
    if (!make_map(&p->mapS_A, p->S16, p->N, p->kpad, TBM, bf16)) return cudaErrorInvalidValue;
    if (!make_map(&p->mapS_B, p->S16, p->N, p->kpad, TBN, bf16)) return cudaErrorInvalidValue;
    if (!make_map(&p->mapP_A, p->A16, p->N, p->kpad, TBM, bf16)) return cudaErrorInvalidValue;
    return cudaSuccess;
}

cudaError_t launch_tc_prep(dd_plan_s* p, cudaStream_t s) {
    const int64_t N = p->N;
    const int n = p->n;
    const bool bf16 = p->opt.precision == DD_TC_BF16;
    const int gN = (int)((N + 255) / 256);
    k_tc_scale<<<1, 32, 0, s>>>(p->stats, bf16 ? 1 : 0);
    k_tc_rowconst<<<gN, 256, 0, s>>>(p->mu_w, p->c_w, p->sigpos, N, n, p->colmu, p->colc, p->rowmu, p->rowc,
                                     p->rowsc, p->ctrl);
    const double u_in = bf16 ? 0.00390625 : 0.00048828125;
    k_tc_rowbound<<<gN, 256, 0, s>>>(p->rowsc, p->rowc, p->rowmu, N, n, u_in, p->stats, p->P2 + p->m, p->ctrl,
                                     p->alpha, p->gam, p->q2);
    const int64_t threads = N * (p->kpad / 8);
    const int g = (int)((threads + 255) / 256);
    if (bf16)
        k_build_S<__nv_bfloat16><<<g, 256, 0, s>>>(p->t64, p->mu_w, p->sig, N, n, p->kpad, p->stats,
                                                   reinterpret_cast<__nv_bfloat16*>(p->S16));
    else
        k_build_S<__half><<<g, 256, 0, s>>>(p->t64, p->mu_w, p->sig, N, n, p->kpad, p->stats,
                                            reinterpret_cast<__half*>(p->S16));
    p->launches += 4;
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(dd_plan_s* p, ListRef L, cudaStream_t s) {
    const int64_t threads = p->N * (p->kpad / 8);
    const int g = (int)((threads + 255) / 256);
    k_gather_rows<<<g, 256, 0, s>>>(L, p->sigpos, reinterpret_cast<const uint4*>(p->S16), p->kpad,
                                    reinterpret_cast<uint4*>(p->A16));
    p->launches++;
    return cudaGetLastError();
}

cudaError_t launch_scan_tc(dd_plan_s* p, const TcArgs& a, bool a_packed, cudaStream_t s) {
    const size_t smem = tc_smem_bytes(p->kpad);
    cudaError_t e = cudaFuncSetAttribute(k_scan_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_scan_tc<<<p->sm_count, kTcThreads, smem, s>>>(a_packed ? p->mapP_A : p->mapS_A, p->mapS_B, a);
    return cudaGetLastError();
}

}  // namespace dd
