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
// Roles (352 threads, one CTA per SM, persistent):
//   warp 0         : scheduler -- claims work items, loads their rows, skips
//                    items whose rows are all abandoned, publishes the rest
//   warp 1         : TMEM allocation (512 columns = two 128x256 FP32 buffers);
//                    lane 0 issues the UMMAs and commits them to mbarriers
//   warps 2-9      : epilogue, two warps per 32-lane TMEM quarter (TMEM lane =
//                    tile row), each taking half of the tile's columns
//   warp 10 lane 0 : TMA producer (operand k-chunks through a ring of stages,
//                    per-column constants by bulk copy)
// All mbarrier waits are bounded with %globaltimer; on expiry the CTA records
// DD_ETIMEOUT in the control block, drains and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cmath>
#include <cuda_fp16.h>

#include "dd_internal.cuh"
#include "tc_ptx.cuh"

namespace dd {
namespace {

constexpr int TBM = 128;
constexpr int TBN = 256;
constexpr int TKA = kTcAtom;  // 16-bit elements per 128-byte swizzle atom
constexpr int kABytesPerAtom = TBM * 128;  // 16 KB
constexpr int kBBytesPerAtom = TBN * 128;  // 32 KB

constexpr int kStageBytes = kABytesPerAtom + kBBytesPerAtom;  // one k-chunk of A and B: 48 KB
constexpr int kStages = 4;
// band mode loads no separate A operand (its rows lie inside the B tile): the
// same bytes hold six B-only stages, so more of the operand stream is in flight
constexpr int kStagesBand = kStages * kStageBytes / kBBytesPerAtom;  // 6
constexpr int kMaxStages = kStagesBand;
constexpr int kItemRing = 4;
constexpr int kEpiWarps = 8;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kTcThreadsV2 = 96 + kEpiThreads;  // scheduler, MMA, 8 epilogue warps, TMA producer

constexpr int kColSlots = 4;
constexpr int kColPad = kTcColPad;  // padding of the per-column constant array on each side
static_assert(kColPad == TBN, "the column constants are padded by one B tile");

struct ItemDesc {
    int rt, pa, pb, dir, nct;  // nct < 0: no more items
    int pad[3];
    float4 row[TBM];           // per tile row: (sqrt(n) mu, c, running minimum, index bits)
};

struct TcHdr {
    unsigned long long b_full[kMaxStages];
    unsigned long long b_empty[kMaxStages];
    unsigned long long acc_full[2];
    unsigned long long acc_empty[2];
    unsigned long long col_full[kColSlots];
    unsigned long long col_empty[kColSlots];
    unsigned long long it_full[kItemRing];
    unsigned long long it_empty[kItemRing];
    uint32_t tmem_base;
    int abort;
    int pad[2];
    ItemDesc items[kItemRing];
    float4 col[kColSlots][TBN];  // per tile column: (sqrt(n) mu, c or +inf, index bits, 0)
};

__device__ __forceinline__ float bound_F(float D, float alpha, float gam, float q2, float beta) {
    return alpha + beta * D + gam * sqrtf(fmaxf(D, 0.f) + q2);
}

__device__ __forceinline__ void item_geometry(const TcArgs& a, int item, int RT, int nseg0, int pos0, int& rt, int& pa,
                                              int& pb, int& dir) {
    if (a.mode == 2) {
        const int s_rank = item / RT;
        rt = item % RT;
        const int4 r = a.ranges[rt];
        pa = pb = 0;
        dir = 1;
        if (s_rank >= r.w) return;
        const int side = s_rank & 1, idx = s_rank >> 1;
        if (side == 0) {
            pa = r.z + idx * a.seg_cols;
            pb = min(pa + a.seg_cols, r.y);
        } else {
            pb = r.z - idx * a.seg_cols;
            pa = max(pb - a.seg_cols, r.x);
            dir = -1;
        }
    } else if (a.mode == 3) {
        // band: the row tile at positions [q0, q0 + 128) of the mean order (q0 = pos0 + 128 rt)
        // against the 256 columns [q0 - 64, q0 + 192) around it (the A rows lie inside that B tile)
        rt = item;
        pa = pos0 + rt * TBM - (TBN - TBM) / 2;
        pb = pa + TBN;
        dir = 1;
    } else {
        // column-segment major: concurrent CTAs share the same operand columns through L2
        const int sg = item / RT;
        rt = item % RT;
        pa = sg * a.seg_cols;
        pb = min(pa + a.seg_cols, a.N);
        dir = 1;
    }
}

// Roles: warp 0 schedules work items and issues the TMA loads (lane 0);
// warp 1 owns the tensor memory and issues the UMMAs (lane 0); warps 2..9
// are the epilogue (two warps per 32-lane TMEM quarter, each taking half of
// a tile's 256 columns).  Work items flow from warp 0 to the others through
// a ring of descriptors; operand k-chunks through a ring of stages; tiles
// through two TMEM accumulators.  Nothing waits on an unbounded barrier.
//
// kBatch: the rows of each list tile belong to one series of a fused batch
// (batch.cu) and are tested against that series' own best-so-far,
// a.sbsf[a.tser[tile]], instead of the control block's.
template <bool kBatch>
__global__ void __launch_bounds__(kTcThreadsV2, 1)
    k_scan_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, TcArgs a) {
    extern __shared__ unsigned char smraw[];
    const uint32_t base_u32 = smem_u32(smraw);
    const uint32_t pad = (1024u - (base_u32 & 1023u)) & 1023u;
    unsigned char* stages = smraw + pad;
    TcHdr& h = *reinterpret_cast<TcHdr*>(stages + kStages * kStageBytes);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const Ctrl* ctrl = a.ctrl;
    if (ctrl->nonfinite || ctrl->degenerate || ctrl->err) return;  // an earlier wave failed: fail fast
    const int cnt = *a.rows.cnt_dev;
    const int off = a.rows.off_dev ? *a.rows.off_dev : 0;
    if (blockIdx.x == 0 && tid == 0 && a.wave >= 0) a.ctrl->wave_rows[a.wave] = cnt;
    const int RT = (cnt + TBM - 1) / TBM;
    if (RT <= 0) return;
    // a list that is a slice of the mean order (a_direct) addresses its operand rows and
    // column constants by position: row r of the list is position pos0 + r
    const int pos0 = a.a_direct ? a.a_row0 + off : 0;
    long long items;
    int nseg0 = 1;
    if (a.mode == 2) {
        const int smax = *a.smax;
        if (smax <= 0) return;
        items = (long long)RT * smax;
    } else if (a.mode == 3) {
        items = RT;
    } else {
        nseg0 = (a.N + a.seg_cols - 1) / a.seg_cols;
        items = (long long)RT * nseg0;
    }

    if (tid == 0) {
        for (int s = 0; s < kMaxStages; s++) {
            mbar_init(&h.b_full[s], 1);
            mbar_init(&h.b_empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&h.acc_full[b], 1);
            mbar_init(&h.acc_empty[b], kEpiThreads);
        }
        for (int c = 0; c < kColSlots; c++) {
            mbar_init(&h.col_full[c], 1);
            mbar_init(&h.col_empty[c], kEpiThreads);
        }
        for (int r = 0; r < kItemRing; r++) {
            mbar_init(&h.it_full[r], 1);
            mbar_init(&h.it_empty[r], 2 + kEpiThreads);  // TMA producer, MMA issuer, epilogue threads
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
    const int n = a.n;
    const int nka = a.nka;
    const bool band = a.mode == 3;
    const int nst = band ? kStagesBand : kStages;              // stages in the ring
    const int sbytes = band ? kBBytesPerAtom : kStageBytes;    // bytes per stage
    const int boff = band ? 0 : kABytesPerAtom;                // B operand offset in a stage

    const int tma_warp = 2 + kEpiWarps;
    if (warp == 0) {
        // ---------------- scheduler: work items, rows, alive check ----------------
        // Items are claimed kClaim at a time; the row loads of a whole batch are
        // issued together and the next claim is in flight while the batch is
        // published, so the global-memory latency is paid once per batch.
        constexpr int kClaim = 4;
        // short waves, and every wave's last items, are claimed one at a time so
        // that every CTA gets work and the CTAs finish together
        const long long tail = (long long)gridDim.x * kClaim * 2;
        int claim = items >= tail ? kClaim : 1;
        int ring = 0;
        uint32_t rph = 0;
        unsigned long long pairs = 0, nrun = 0;
        bool ok = true;
        // Lower-bound full scans (mode 2) also skip a segment when no row of the
        // tile can still be lowered by it: every column j of the segment has
        // d^2 >= n (mu_i - mu_j)^2 and that exceeds the row's current upper
        // bound.  The segment's sqrt(n) mu range comes from its end columns
        // widened by one mean bin (columns are sorted by bin, not by exact mean).
        const bool seg_check = a.mode == 2 && a.abandon;
        // local waves (mode 2 with local_k > 0): row i only needs the columns
        // within local_k positions of its own place in the mean order
        const bool local = a.mode == 2 && a.local_k > 0;
        const float snw = sqrtf((float)n) * (float)a.stats[7] * 1.001f;
        int base = 0;
        if (lane == 0) base = atomicAdd(&a.ctrl->work[a.work_slot], claim);
        base = __shfl_sync(0xffffffffu, base, 0);
        while (ok && base >= 0 && base < items && !*abort) {
            int rt[kClaim], pa[kClaim], pb[kClaim], dir[kClaim];
            float4 rowd[kClaim][4];  // per row: (sqrt(n) mu, c, running minimum, orig index bits)
            float segL[kClaim], segH[kClaim], bsfv[kClaim];
            const float bsf = __uint_as_float(*((volatile const unsigned*)&ctrl->bsf));
#pragma unroll
            for (int b = 0; b < kClaim; b++) {
                const long long item = b < claim ? (long long)base + b : items;
                rt[b] = 0;
                pa[b] = pb[b] = 0;
                dir[b] = 1;
                if (item < items) item_geometry(a, (int)item, RT, nseg0, pos0, rt[b], pa[b], pb[b], dir[b]);
                // the row tile is known without the column range: load its rows in parallel with it
                const int rtb = item < items ? (a.mode == 3 ? (int)item : (int)(item % RT)) : RT;
                bsfv[b] = bsf;
                if (kBatch && rtb < RT) bsfv[b] = __uint_as_float(*((volatile const unsigned*)(a.sbsf + a.tser[rtb])));
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int r = rtb * TBM + q * 32 + lane;
                    rowd[b][q] = make_float4(0.f, 0.f, INFINITY, __int_as_float(-1));
                    if (r < cnt) {
                        if (a.a_direct) {  // a slice of the mean order: row r is column pos0 + r
                            const float4 cd = a.coldat[kColPad + pos0 + r];  // (sqrt(n) mu, c, index bits, 0)
                            rowd[b][q] = make_float4(cd.x, cd.y, INFINITY, cd.z);
                        } else
                            rowd[b][q].w = __int_as_float(a.rows.base[off + r]);
                    }
                }
                segL[b] = -INFINITY;
                segH[b] = INFINITY;
                if (seg_check && pa[b] < pb[b]) {
                    segL[b] = a.coldat[kColPad + pa[b]].x - snw;
                    segH[b] = a.coldat[kColPad + pb[b] - 1].x + snw;
                }
            }
            // the error bound of a row is needed to test it against a best-so-far or a lower bound
            bool any[kClaim];
#pragma unroll
            for (int b = 0; b < kClaim; b++) {
                const bool need_bound = seg_check || local || (a.abandon && bsfv[b] > 0.f);
                const bool up = dir[b] > 0;
                bool fin = true;  // no live row needs this segment or any farther one on its side
                any[b] = !a.abandon && !local;
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int i = __float_as_int(rowd[b][q].w);
                    if (i < 0 || pa[b] >= pb[b]) {
                        rowd[b][q] = make_float4(0.f, 0.f, INFINITY, __int_as_float(-1));
                        continue;
                    }
                    const float D = __uint_as_float(*((volatile const unsigned*)(a.rmin + i)));
                    rowd[b][q].z = D;
                    if (!a.a_direct) {
                        rowd[b][q].x = a.rowmu[i];
                        rowd[b][q].y = a.rowc[i];
                    }
                    if (!a.abandon && !local) continue;
                    if (!need_bound) {  // nothing has completed: every row is live and needs every column
                        any[b] = true;
                        fin = false;
                        continue;
                    }
                    float R = D + bound_F(D, a.alpha[i], a.gam[i], a.q2[i], a.beta);
                    if (a.r32) R = fminf(R, __uint_as_float(a.r32[i]));
                    // a row whose upper bound is below the best-so-far stays below it
                    if (a.abandon && R < bsfv[b]) continue;
                    bool need = true, need_far = true;
                    if (seg_check) {
                        const float x = rowd[b][q].x;
                        const float lim = sqrtf(R) * 1.001f + 1e-5f * (fabsf(x) + fabsf(segL[b]) + fabsf(segH[b]));
                        const float dd = fmaxf(fmaxf(segL[b] - x, x - segH[b]), 0.f);
                        // every column at or beyond the segment (on its side) lies past segL / segH
                        const float df = fmaxf(up ? segL[b] - x : x - segH[b], 0.f);
                        need = !(dd > lim);  // NaN -> needed
                        need_far = !(df > lim);
                    }
                    if (local) {
                        const int qi = a.sigpos[i];
                        need = need && pa[b] <= qi + a.local_k && pb[b] > qi - a.local_k;
                        need_far = need_far && (up ? qi + a.local_k >= pa[b] : qi - a.local_k < pb[b]);
                    }
                    any[b] |= need;
                    fin = fin && !need_far;
                }
                // shrink the tile's column range: later items of this side see an empty segment
                if ((seg_check || local) && pa[b] < pb[b] && __all_sync(0xffffffffu, fin) && lane == 0) {
                    if (up)
                        atomicMin(&a.ranges[rt[b]].y, pa[b]);
                    else
                        atomicMax(&a.ranges[rt[b]].x, pb[b]);
                }
            }
            int nbase = 0;
            const int nclaim = items - (long long)base > tail ? kClaim : 1;
            if (lane == 0) nbase = atomicAdd(&a.ctrl->work[a.work_slot], nclaim);
#pragma unroll
            for (int b = 0; b < kClaim; b++) {
                if (!__any_sync(0xffffffffu, any[b] && pa[b] < pb[b])) continue;
                int nvr = 0;
#pragma unroll
                for (int q = 0; q < 4; q++) nvr += __float_as_int(rowd[b][q].w) >= 0 ? 1 : 0;
                nvr = __reduce_add_sync(0xffffffffu, nvr);
                if (lane == 0 && !mbar_wait(&h.it_empty[ring], rph ^ 1u, abort)) ok = false;
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                if (!ok) break;
#pragma unroll
                for (int q = 0; q < 4; q++) h.items[ring].row[q * 32 + lane] = rowd[b][q];
                __threadfence_block();
                __syncwarp();
                if (lane == 0) {
                    pairs += (unsigned long long)nvr * (unsigned long long)(pb[b] - pa[b]);
                    nrun++;
                    ItemDesc& d = h.items[ring];
                    d.rt = rt[b];
                    d.pa = pa[b];
                    d.pb = pb[b];
                    d.dir = dir[b];
                    d.nct = (pb[b] - pa[b] + TBN - 1) / TBN;
                    mbar_arrive(&h.it_full[ring]);
                }
                if (++ring == kItemRing) {  // every lane keeps the ring position
                    ring = 0;
                    rph ^= 1u;
                }
            }
            base = __shfl_sync(0xffffffffu, nbase, 0);
            claim = nclaim;
        }
        if (lane == 0) {
            if (!ok) {
                atomicExch(&a.ctrl->err, DD_ETIMEOUT);
                *abort = 1;
            } else if (base < 0) {
                atomicExch(&a.ctrl->err, DD_ENOTSUP);  // the 32-bit work counter wrapped
            }
            // end marker (bounded wait; on abort the consumers leave on their own)
            if (mbar_wait(&h.it_empty[ring], rph ^ 1u, abort)) {
                h.items[ring].nct = -1;
                mbar_arrive(&h.it_full[ring]);
            }
            if (pairs) atomicAdd(&a.ctrl->pairs, pairs);
            if (a.wave >= 0) {
                if (pairs) atomicAdd(&a.ctrl->wave_pairs[a.wave], pairs);
                if (nrun) atomicAdd(&a.ctrl->wave_items[a.wave], nrun);
            }
        }
        __syncwarp();
    } else if (warp == tma_warp) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            int stage = 0, ring = 0, cslot = 0;
            uint32_t sph = 0, rph = 0, cph = 0;
            bool ok = true;
            for (;;) {
                if (!mbar_wait(&h.it_full[ring], rph, abort)) {
                    ok = false;
                    break;
                }
                const int rt = h.items[ring].rt, pa = h.items[ring].pa, pb = h.items[ring].pb;
                const int dir = h.items[ring].dir, nct = h.items[ring].nct;
                mbar_arrive(&h.it_empty[ring]);
                if (++ring == kItemRing) {
                    ring = 0;
                    rph ^= 1u;
                }
                if (nct < 0) break;
                const int arow = rt * TBM + pos0;
                for (int ct = 0; ct < nct && ok; ct++) {
                    const int p0 = dir > 0 ? pa + ct * TBN : pb - (ct + 1) * TBN;
                    // per-column constants of the tile (padded array: p0 >= -TBN, p0 + TBN <= N + TBN)
                    if (!mbar_wait(&h.col_empty[cslot], cph ^ 1u, abort)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&h.col_full[cslot], (uint32_t)(TBN * sizeof(float4)));
                    bulk_load(&h.col[cslot][0], a.coldat + kColPad + p0, (uint32_t)(TBN * sizeof(float4)),
                              &h.col_full[cslot]);
                    if (++cslot == kColSlots) {
                        cslot = 0;
                        cph ^= 1u;
                    }
                    for (int ka = 0; ka < nka; ka++) {
                        if (!mbar_wait(&h.b_empty[stage], sph ^ 1u, abort)) {
                            ok = false;
                            break;
                        }
                        unsigned char* st = stages + stage * sbytes;
                        // a.stall (fault injection for tests): arm the stage but issue no copy, so the
                        // waits on it expire and the launch ends with DD_ETIMEOUT
                        if (band) {  // A rows come from inside the B tile
                            mbar_expect_tx(&h.b_full[stage], (uint32_t)kBBytesPerAtom);
                        } else {
                            mbar_expect_tx(&h.b_full[stage], (uint32_t)kStageBytes);
                            if (!a.stall) tma_load_3d(st, &mapA, &h.b_full[stage], arow, ka);
                        }
                        if (!a.stall) tma_load_3d(st + boff, &mapB, &h.b_full[stage], p0, ka);
                        if (++stage == nst) {
                            stage = 0;
                            sph ^= 1u;
                        }
                    }
                }
                if (!ok) break;
            }
            if (!ok) {
                atomicExch(&a.ctrl->err, DD_ETIMEOUT);
                *abort = 1;
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- UMMA issuer ----------------
        if (lane == 0) {
            int stage = 0, ring = 0, tb = 0;
            uint32_t sph = 0, rph = 0;
            uint32_t aph[2] = {0u, 0u};
            bool ok = true;
            for (;;) {
                if (!mbar_wait(&h.it_full[ring], rph, abort)) {
                    ok = false;
                    break;
                }
                const ItemDesc d = h.items[ring];
                mbar_arrive(&h.it_empty[ring]);
                if (++ring == kItemRing) {
                    ring = 0;
                    rph ^= 1u;
                }
                if (d.nct < 0) break;
                for (int ct = 0; ct < d.nct && ok; ct++) {
                    if (!mbar_wait(&h.acc_empty[tb], aph[tb] ^ 1u, abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dt = tbase + (uint32_t)(tb * TBN);
                    for (int ka = 0; ka < nka; ka++) {
                        if (!mbar_wait(&h.b_full[stage], sph, abort)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t sa = smem_u32(stages + stage * sbytes);
                        // band mode: A = B rows [64, 192), 8 KB into the B tile (a whole number of 1 KB swizzle atoms)
                        const uint64_t ad = sw128_desc(band ? sa + (TBN - TBM) / 2 * 128 : sa);
                        const uint64_t bd = sw128_desc(sa + boff);
#pragma unroll
                        for (int kk = 0; kk < TKA / 16; kk++)
                            umma_f16(dt, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), a.idesc,
                                     (ka | kk) != 0 ? 1u : 0u);
                        umma_commit(&h.b_empty[stage]);
                        if (++stage == nst) {
                            stage = 0;
                            sph ^= 1u;
                        }
                    }
                    if (!ok) break;
                    umma_commit(&h.acc_full[tb]);
                    aph[tb] ^= 1u;
                    tb ^= 1;
                }
                if (!ok) break;
            }
            if (!ok) {
                atomicExch(&a.ctrl->err, DD_ETIMEOUT);
                *abort = 1;
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue (warps 2 .. 2 + kEpiWarps - 1) ----------------
        const int q = warp & 3;            // TMEM lane quarter
        const int half = (warp - 2) >> 2;  // column half of the tile
        const float neg2s = (float)(-2.0 / (a.stats[3] * a.stats[3]));  // s is a power of two: exact
        int ring = 0, tb = 0, cslot = 0;
        uint32_t rph = 0, cph = 0;
        uint32_t aph[2] = {0u, 0u};
        for (;;) {
            bool ok = mbar_wait(&h.it_full[ring], rph, abort);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            const int nct = h.items[ring].nct;
            const float4 rd = h.items[ring].row[q * 32 + lane];
            mbar_arrive(&h.it_empty[ring]);
            if (++ring == kItemRing) {
                ring = 0;
                rph ^= 1u;
            }
            if (nct < 0) break;
            const float rmu = rd.x, rc = rd.y;
            const int ri = __float_as_int(rd.w);
            float Drun = rd.z;
            const float Dlast = Drun;
            for (int ct = 0; ct < nct; ct++) {
                bool okw = mbar_wait(&h.col_full[cslot], cph, abort);
                okw = okw && mbar_wait(&h.acc_full[tb], aph[tb], abort);
                aph[tb] ^= 1u;
                okw = __all_sync(0xffffffffu, okw);  // tcgen05.ld is warp-wide
                if (!okw) {
                    atomicExch(&a.ctrl->err, DD_ETIMEOUT);
                    *abort = 1;
                    break;
                }
                tc_fence_after();
                float m = INFINITY;
                const uint32_t taddr = tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(tb * TBN + half * (TBN / 2));
#pragma unroll 1
                for (int ch = 0; ch < TBN / 2 / 32; ch++) {
                    uint32_t v[32];
                    tmem_ld32(taddr + (uint32_t)(ch * 32), v);
                    tmem_ld_wait();
                    const float4* cdp = &h.col[cslot][half * (TBN / 2) + ch * 32];
#pragma unroll
                    for (int x = 0; x < 32; x++) {
                        const float4 cd = cdp[x];
                        const float dm = rmu - cd.x;
                        float t = fmaf(dm, dm, cd.y);
                        t = fmaf(neg2s, __uint_as_float(v[x]), t);
                        const int j = __float_as_int(cd.z);
                        const bool okc = (unsigned)(j - ri + n - 1) >= (unsigned)(2 * n - 1);
                        m = okc ? fminf(m, t) : m;
                    }
                }
                tc_fence_before();
                mbar_arrive(&h.acc_empty[tb]);
                mbar_arrive(&h.col_empty[cslot]);
                tb ^= 1;
                if (++cslot == kColSlots) {
                    cslot = 0;
                    cph ^= 1u;
                }
                Drun = fminf(Drun, fmaxf(m + rc, 0.f));
            }
            if (ri >= 0 && Drun < Dlast) atomicMin(a.rmin + ri, __float_as_uint(Drun));
            if (*abort) break;
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
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    // resolved once (thread-safe static initialisation: plans are created from several threads)
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeTiledFn>(ptr);
    }();
    return fn;
}

bool make_map(CUtensorMap* map, void* base, int64_t rows, int kpad, int box_rows, bool bf16) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    // [kpad / 64][rows][64] elements: 128-byte rows, one plane per 64-element k-chunk
    cuuint64_t dims[3] = {(cuuint64_t)TKA, (cuuint64_t)rows, (cuuint64_t)(kpad / TKA)};
    cuuint64_t strides[2] = {(cuuint64_t)TKA * 2, (cuuint64_t)rows * TKA * 2};
    cuuint32_t box[3] = {(cuuint32_t)TKA, (cuuint32_t)box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, base, dims,
                    strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

__global__ void k_coldat_pad(float4* coldat, int64_t N) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * kColPad) return;
    const int64_t ix = t < kColPad ? t : N + t;  // [0, pad) and [pad + N, 2 pad + N)
    coldat[ix] = make_float4(0.f, INFINITY, __int_as_float(-(1 << 30)), 0.f);
}

cudaError_t tc_init_plan(dd_plan_s* p, cudaStream_t s) {
    k_coldat_pad<<<(2 * kColPad + 255) / 256, 256, 0, s>>>(p->coldat, p->N);
    return cudaGetLastError();
}

size_t tc_smem_bytes(int kpad) {
    (void)kpad;
    return 1024 + (size_t)kStages * kStageBytes + sizeof(TcHdr);
}

int tc_stages(int kpad) {
    (void)kpad;
    return kStages;
}

bool tc_supported(int n) {
    return n >= 1 && n <= (1 << 16);
}

cudaError_t tc_make_maps(dd_plan_s* p) {
    const bool bf16 = p->opt.precision == DD_TC_BF16;
    if (!make_map(&p->mapS_A, p->S16, p->N, p->kpad, TBM, bf16)) return cudaErrorInvalidValue;
    if (!make_map(&p->mapS_B, p->S16, p->N, p->kpad, TBN, bf16)) return cudaErrorInvalidValue;
    if (!make_map(&p->mapP_A, p->A16, p->N, p->kpad, TBM, bf16)) return cudaErrorInvalidValue;
    return cudaSuccess;
}

cudaError_t launch_scan_tc(dd_plan_s* p, const TcArgs& a, bool a_packed, cudaStream_t s) {
    const size_t smem = tc_smem_bytes(p->kpad);
    const bool batch = a.sbsf != nullptr;
    cudaError_t e = cudaFuncSetAttribute(batch ? k_scan_tc<true> : k_scan_tc<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (batch)
        k_scan_tc<true><<<p->sm_count, kTcThreadsV2, smem, s>>>(a_packed ? p->mapP_A : p->mapS_A, p->mapS_B, a);
    else
        k_scan_tc<false><<<p->sm_count, kTcThreadsV2, smem, s>>>(a_packed ? p->mapP_A : p->mapS_A, p->mapS_B, a);
    return cudaGetLastError();
}

}  // namespace dd
