// scan_fp32.cu -- distance tiles in the plain FP32 form (Eq. 1 squared,
// direct differences sum_k (x_k - y_k)^2 on the CUDA cores), the inner loops
// of Algorithms 3 and 4 with early abandon against the best-so-far.
//
// One work item = a tile of 128 rows of a row list x a segment of a wave's
// columns.  The CTA walks the segment's 128-column tiles in order; after each
// tile it publishes the rows' running minima (atomicMin on float bits) and,
// when abandoning, stops as soon as every row of the tile has a distance
// strictly below the best-so-far (such a row cannot be the discord).
// Work items are handed out dynamically through an atomic counter (the
// GPU counterpart of the paper's dynamic OpenMP schedule).
//
// Column sets: see ColSpec (mean-order ranges, word buckets, lower-bound
// segments, time-local windows).  In a Gram-form plan this kernel runs the
// time-local and settle waves: it then tests rows against the Gram bound and
// publishes rigorous FP32 upper bounds to r32 (see TcBound) instead of plain
// minima.
//
// Tile arithmetic: 256 threads, each an 8x8 register micro-tile of
// (row, column) pairs in packed FP32 pairs (one f32x2 subtract and one f32x2
// FMA per two pairs and k); k is staged through shared memory in chunks of 32 with
// cp.async double buffering; rows and columns are gathered by index, each
// being n consecutive values of the normalised series t^ (FP32).
#include "dd_internal.cuh"

namespace dd {
namespace {

constexpr int BN = kF32BN, BK = kF32BK, NT = kF32Threads;

// BM rows per tile: 128 (every wave of a search), or 64 / 32 (the fused batch's
// settle tiles, which hold one series' few candidates).  A thread's micro-tile is
// BM / 16 rows x 8 columns.
template <int BM>
struct __align__(16) F32Smem {
    static constexpr int SROW = BM + 4;  // floats per k-row of the transposed row tile (16-B aligned)
    static constexpr int SCOL = BN + 4;
    float a[2][BK][SROW];
    float b[2][BK][SCOL];
    int row[BM];
    int col[BN];
    float rmin[BM];
    float last[BM];
    int item;
    unsigned bsf;
    int nvalid_rows;
    int pad;
};

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, bool pred) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    int sz = pred ? 4 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Stage k-chunk [k0, k0+BK) of the tile's rows and columns (transposed).
template <int BM>
__device__ __forceinline__ void stage_chunk(F32Smem<BM>& sm, int buf, const float* __restrict__ t32, int k0, int n) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = k0 + lane;
    const bool kin = k < n;
#pragma unroll 4
    for (int q = 0; q < BM / 8; q++) {
        const int r = warp + 8 * q;
        const int ri = sm.row[r];
        const bool ok = kin && ri >= 0;
        cp_async4(&sm.a[buf][lane][r], ok ? (const void*)(t32 + ri + k) : (const void*)t32, ok);
    }
#pragma unroll 4
    for (int q = 0; q < BN / 8; q++) {
        const int c = warp + 8 * q;
        const int cj = sm.col[c];
        const bool ok = kin && cj >= 0;
        cp_async4(&sm.b[buf][lane][c], ok ? (const void*)(t32 + cj + k) : (const void*)t32, ok);
    }
}

// Packed FP32 pairs (sm_100+ f32x2 arithmetic): every lane of a pair is rounded
// exactly as the scalar instruction would round it, so a pair's distance is the
// same sum of the same terms in the same k order; one instruction does two.
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t f2_dup(float x) {
    f2_t r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b) {
    f2_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
// c + d * d, lane by lane
__device__ __forceinline__ f2_t f2_fma_sq(f2_t d, f2_t c) {
    f2_t r;
    asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(r) : "l"(d), "l"(c));
    return r;
}
__device__ __forceinline__ float f2_lo(f2_t v) { return __uint_as_float((unsigned)(v & 0xffffffffull)); }
__device__ __forceinline__ float f2_hi(f2_t v) { return __uint_as_float((unsigned)(v >> 32)); }

// Rigorous upper bound on the exact squared distance d^2 (FP64 series) of a
// pair whose FP32 value is e: inputs rounded to FP32 (|t^| <= M), FP32
// differences, FMA accumulation of n terms -- the same bound, doubled, as the
// FP32 screen of the exact rescoring.
__device__ __forceinline__ float fp32_upper(float e, float n, float M) {
    const float u = 5.9604644775390625e-08f;  // 2^-24
    const float gn = n * u / (1.f - n * u);
    const float mu6 = 6.f * u * M;
    return e + 2.f * ((gn + 4.f * u) * e + 8.f * u * M * sqrtf(n * e) + n * mu6 * mu6) + 1e-30f;
}

template <int BM>
__global__ void __launch_bounds__(NT, 2) k_scan_fp32(ScanArgs a) {
    constexpr int RI = BM / 16;  // rows of a thread's micro-tile
    extern __shared__ __align__(16) unsigned char smraw[];
    F32Smem<BM>& sm = *reinterpret_cast<F32Smem<BM>*>(smraw);
    const Ctrl* ctrl = a.ctrl_ro;
    if (ctrl->nonfinite || ctrl->degenerate) return;
    const int cnt = *a.rows.cnt_dev;
    if (cnt <= a.min_rows) return;  // gated off on the device (the list is too short to be worth a wave)
    const int off = a.rows.off_dev ? *a.rows.off_dev : 0;
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.wave >= 0) a.ctrl->wave_rows[a.wave] = cnt;
    const int RT = (cnt + BM - 1) / BM;
    if (RT <= 0) return;
    const int mode = a.col.mode;
    // work decomposition
    long long items;
    int nseg = 1, CT = 0, V = 0;
    if (mode == 2) {
        const int smax = *a.smax;
        if (smax <= 0) return;
        items = (long long)RT * smax;
    } else {
        if (mode == 0) {
            const int hi = a.col.v_hi < a.N ? a.col.v_hi : a.N;
            V = hi - a.col.v_lo;
        } else {
            V = mode == 4 ? 2 * a.col.local_cols : a.col.local_cols;
        }
        if (V <= 0) return;
        CT = (V + BN - 1) / BN;
        nseg = (a.target_items + RT - 1) / RT;
        int maxseg = CT / (a.min_seg_tiles > 0 ? a.min_seg_tiles : 1);
        if (maxseg < 1) maxseg = 1;
        if (nseg > maxseg) nseg = maxseg;
        if (nseg < 1) nseg = 1;
        items = (long long)RT * nseg;
    }

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int n = a.n;
    const int nk = (n + BK - 1) / BK;
    const bool assist = a.r32 != nullptr;
    const float nf = (float)n;
    const float tmax = assist ? (float)a.stats[2] : 0.f;
    unsigned long long pairs = 0, nrun = 0;

    for (;;) {
        __syncthreads();  // the previous item is done with sm.item and the tiles
        if (tid == 0) sm.item = atomicAdd(&a.ctrl->work[a.work_slot], 1);
        __syncthreads();
        const int item = sm.item;
        if (item < 0 || item >= items) {
            // a negative claim: the 32-bit work counter wrapped (more than 2^31 items)
            if (item < 0 && tid == 0) atomicExch(&a.ctrl->err, DD_ENOTSUP);
            break;
        }
        // item -> row tile + column tiles
        int rt, ct0, ct1;
        int pa = 0, pb = 0, dir = 1;  // mode 2: positions [pa, pb) of sig, walked up (dir 1) or down
        if (mode == 2) {
            const int s_rank = item / RT;
            rt = item % RT;
            const int4 r = a.ranges[rt];
            if (s_rank >= r.w) continue;  // uniform: the whole block skips
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
            if (pa >= pb) continue;
            ct0 = 0;
            ct1 = (pb - pa + BN - 1) / BN;
        } else {
            rt = item / nseg;
            const int sg = item % nseg;
            ct0 = (int)(((long long)sg * CT) / nseg);
            ct1 = (int)(((long long)(sg + 1) * CT) / nseg);
        }

        if (tid < BM) {
            const int r = rt * BM + tid;
            const int ri = r < cnt ? a.rows.base[off + r] : -1;
            sm.row[tid] = ri;
            // assisting a Gram-form plan, the tile keeps plain FP32 minima (from +inf) and
            // publishes their upper bounds to r32
            const float v = (ri >= 0 && !assist) ? __uint_as_float(a.rmin[ri]) : INFINITY;
            sm.rmin[tid] = v;
            sm.last[tid] = v;
        }
        __syncthreads();
        // same-word neighbourhood of the tile's first row (mode 1)
        int bs = 0, bsz = 1, startoff = 0, L = V;
        if (mode == 1) {
            const int r0 = sm.row[0];
            const int h = a.code[r0];
            bs = a.word_start[h];
            bsz = a.hist[h];
            const int p0 = a.pos_of[r0];
            startoff = (p0 - bs + bsz / 2) % bsz;
            L = a.col.local_cols < bsz ? a.col.local_cols : bsz;
        }
        const int nvr = __syncthreads_count(tid < BM && sm.row[tid] >= 0);
        // time-local neighbourhood (mode 4): the tile's rows are in time order
        const int t_first = sm.row[0], t_last = sm.row[nvr > 0 ? nvr - 1 : 0];
        bool ran = false;

        for (int ct = ct0; ct < ct1; ct++) {
            if (a.abandon) {
                bool alive = false;
                if (tid < BM) {
                    const int ri = sm.row[tid];
                    if (ri >= 0) {
                        const float g = __uint_as_float(*((volatile const unsigned*)(a.rmin + ri)));
                        const float bsf = __uint_as_float(
                            *((volatile const unsigned*)(a.sbsf ? a.sbsf + a.tser[rt] : &ctrl->bsf)));
                        const float mn = fminf(sm.rmin[tid], g);
                        alive = assist ? !(fminf(row_ub(a.tb, ri, g), fp32_upper(sm.rmin[tid], nf, tmax)) < bsf)
                                       : !(mn < bsf);
                    }
                }
                if (!__syncthreads_or(alive)) break;
            }
            int valid_col = 0;
            if (tid < BN) {
                int cj = -1;
                if (mode == 0) {
                    const int v = a.col.v_lo + ct * BN + tid;
                    if (v < a.col.v_lo + V) cj = a.order[a.N - 1 - v];
                } else if (mode == 1) {
                    const int v = ct * BN + tid;
                    if (v < L) cj = a.order[bs + (startoff + v) % bsz];
                } else if (mode == 4) {
                    const int v = ct * BN + tid;
                    const int K = a.col.local_cols;
                    if (v < V) {
                        const int j = v < K ? t_first - n - K + 1 + v : t_last + n + (v - K);
                        cj = (j >= 0 && j < a.N) ? j : -1;
                    }
                } else {
                    const int p = dir > 0 ? pa + ct * BN + tid : pb - 1 - ct * BN - tid;
                    if (p >= pa && p < pb) cj = a.sig[p];
                }
                sm.col[tid] = cj;
                valid_col = cj >= 0;
            }
            const int nvc = __syncthreads_count(valid_col);
            if (nvc == 0) continue;
            pairs += (unsigned long long)nvr * (unsigned long long)nvc;
            if (!ran) {
                ran = true;
                nrun++;
            }

            // acc2[i][q] holds columns 2q, 2q + 1 of row i
            f2_t acc2[RI][4];
#pragma unroll
            for (int i = 0; i < RI; i++)
#pragma unroll
                for (int q = 0; q < 4; q++) acc2[i][q] = 0ull;

            stage_chunk(sm, 0, a.t32, 0, n);
            cp_async_commit();
            for (int kc = 0; kc < nk; kc++) {
                const int buf = kc & 1;
                if (kc + 1 < nk) {
                    stage_chunk(sm, buf ^ 1, a.t32, (kc + 1) * BK, n);
                    cp_async_commit();
                    cp_async_wait<1>();
                } else {
                    cp_async_wait<0>();
                }
                __syncthreads();
#pragma unroll 8
                for (int kk = 0; kk < BK; kk++) {
                    float x[RI];
                    if constexpr (BM == 128) {
                        const float4 a0 = *reinterpret_cast<const float4*>(&sm.a[buf][kk][ty * 4]);
                        const float4 a1 = *reinterpret_cast<const float4*>(&sm.a[buf][kk][64 + ty * 4]);
                        x[0] = a0.x; x[1] = a0.y; x[2] = a0.z; x[3] = a0.w;
                        x[4] = a1.x; x[5] = a1.y; x[6] = a1.z; x[7] = a1.w;
                    } else if constexpr (BM == 64) {
                        const float4 a0 = *reinterpret_cast<const float4*>(&sm.a[buf][kk][ty * 4]);
                        x[0] = a0.x; x[1] = a0.y; x[2] = a0.z; x[3] = a0.w;
                    } else {
                        const float2 a0 = *reinterpret_cast<const float2*>(&sm.a[buf][kk][ty * 2]);
                        x[0] = a0.x; x[1] = a0.y;
                    }
                    const ulonglong2 b0 = *reinterpret_cast<const ulonglong2*>(&sm.b[buf][kk][tx * 4]);
                    const ulonglong2 b1 = *reinterpret_cast<const ulonglong2*>(&sm.b[buf][kk][64 + tx * 4]);
                    const f2_t y2[4] = {b0.x, b0.y, b1.x, b1.y};
#pragma unroll
                    for (int i = 0; i < RI; i++) {
                        const f2_t xx = f2_dup(x[i]);
#pragma unroll
                        for (int q = 0; q < 4; q++) acc2[i][q] = f2_fma_sq(f2_sub(xx, y2[q]), acc2[i][q]);
                    }
                }
                __syncthreads();
            }
            // exclusion zone |i - j| < n, row minima over the 128 columns
            int cjr[8];
#pragma unroll
            for (int j = 0; j < 8; j++) cjr[j] = sm.col[j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4)];
#pragma unroll
            for (int i = 0; i < RI; i++) {
                const int r = BM == 128 ? (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4)) : ty * RI + i;
                const int ri = sm.row[r];
                float mn = INFINITY;
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    const int d = ri - cjr[j];
                    const bool ok = cjr[j] >= 0 && (d >= n || d <= -n);
                    const float v = (j & 1) ? f2_hi(acc2[i][j >> 1]) : f2_lo(acc2[i][j >> 1]);
                    mn = ok ? fminf(mn, v) : mn;
                }
                mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, 1));
                mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, 2));
                mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, 4));
                mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, 8));
                if (tx == 0 && mn < sm.rmin[r]) sm.rmin[r] = mn;
            }
            __syncthreads();
            if (a.abandon && tid < BM) {
                const int ri = sm.row[tid];
                const float v = sm.rmin[tid];
                if (ri >= 0 && v < sm.last[tid]) {
                    if (assist)
                        atomicMin(a.r32 + ri, __float_as_uint(fp32_upper(v, nf, tmax)));
                    else
                        atomicMin(a.rmin + ri, __float_as_uint(v));
                    sm.last[tid] = v;
                }
            }
        }
        if (tid < BM) {
            const int ri = sm.row[tid];
            const float v = sm.rmin[tid];
            if (ri >= 0 && v < sm.last[tid])
                atomicMin(assist ? a.r32 + ri : a.rmin + ri,
                          __float_as_uint(assist ? fp32_upper(v, nf, tmax) : v));
        }
        __syncthreads();
    }
    if (tid == 0 && pairs) atomicAdd(&a.ctrl->pairs, pairs);
    if (tid == 0 && a.wave >= 0) {
        if (pairs) atomicAdd(&a.ctrl->wave_pairs[a.wave], pairs);
        if (nrun) atomicAdd(&a.ctrl->wave_items[a.wave], nrun);
    }
}

}  // namespace

int scan_fp32_grid(const dd_plan_s* p) { return p->sm_count * 2; }

template <int BM>
cudaError_t launch_bm(const ScanArgs& a, int grid, cudaStream_t s) {
    static std::atomic<int> attr_set{0};
    if (!attr_set.load()) {
        cudaError_t e = cudaFuncSetAttribute(k_scan_fp32<BM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(F32Smem<BM>));
        if (e != cudaSuccess) return e;
        attr_set.store(1);
    }
    k_scan_fp32<BM><<<grid, NT, sizeof(F32Smem<BM>), s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_scan_fp32(const ScanArgs& a, int grid, cudaStream_t s) {
    if (a.bm == 64) return launch_bm<64>(a, grid, s);
    if (a.bm == 32) return launch_bm<32>(a, grid, s);
    if (a.bm != 0 && a.bm != 128) return cudaErrorInvalidValue;
    return launch_bm<128>(a, grid, s);
}

}  // namespace dd
