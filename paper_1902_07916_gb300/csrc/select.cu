// Kernels (b) and (c): per-cell statistics and the level threshold, cell
// selection with an ordered block-scan compaction into the next level's work
// list, and the compensated final reduction.  All run on a fixed grid
// (kSelGrid CTAs) of which a level uses as many as its size needs
// (active_ctas), each owning one contiguous chunk of the level's cells; the
// count depends on the level's size only, so results are bit-reproducible on
// any GPU.  Grid-wide steps (threshold, scan of the per-CTA counts, the
// level's accepted sums) are done by the last CTA to arrive at a ticket
// counter; no CTA ever waits on another.
#include <float.h>
#include <math.h>

#include <string>

#include "zmc_device.cuh"
#include "zmc_internal.h"

namespace zmc {

namespace {

// Chan et al. pairwise merge of (count, mean, M2) summaries.
struct Moments {
    double n, mean, m2;
};

__device__ __forceinline__ Moments merge(Moments a, Moments b) {
    if (a.n == 0.0) return b;
    if (b.n == 0.0) return a;
    const double n = a.n + b.n;
    const double delta = b.mean - a.mean;
    Moments r;
    r.n = n;
    r.mean = a.mean + delta * (b.n / n);
    r.m2 = a.m2 + b.m2 + delta * delta * (a.n * b.n / n);
    return r;
}

__device__ __forceinline__ Moments shfl_moments(Moments v, int o) {
    Moments r;
    r.n = __shfl_xor_sync(0xFFFFFFFFu, v.n, o);
    r.mean = __shfl_xor_sync(0xFFFFFFFFu, v.mean, o);
    r.m2 = __shfl_xor_sync(0xFFFFFFFFu, v.m2, o);
    return r;
}

// Fixed-order block merge of per-thread moments (blockDim = kSelThreads).
__device__ Moments block_merge(Moments v) {
    __shared__ Moments s[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        Moments w = shfl_moments(v, o);
        v = (lane & o) ? merge(w, v) : merge(v, w);
    }
    if (lane == 0) s[warp] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    if (warp == 0) {
        v = lane < nw ? s[lane] : Moments{0.0, 0.0, 0.0};
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            Moments w = shfl_moments(v, o);
            v = (lane & o) ? merge(w, v) : merge(v, w);
        }
    }
    __syncthreads();
    return v;  // valid in thread 0
}

// Compensated (sum, err) pair.  add() is Neumaier-style via TwoSum.
struct CSum {
    double s, e;
    __device__ __forceinline__ void add(double x) {
        double t, r;
        two_sum(s, x, t, r);
        s = t;
        e += r;
    }
    __device__ __forceinline__ void add(CSum o) {
        double t, r;
        two_sum(s, o.s, t, r);
        s = t;
        e += o.e + r;
    }
};

__device__ CSum block_csum(CSum v) {
    __shared__ CSum s[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        CSum w{__shfl_xor_sync(0xFFFFFFFFu, v.s, o), __shfl_xor_sync(0xFFFFFFFFu, v.e, o)};
        v.add(w);
    }
    if (lane == 0) s[warp] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    if (warp == 0) {
        v = lane < nw ? s[lane] : CSum{0.0, 0.0};
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            CSum w{__shfl_xor_sync(0xFFFFFFFFu, v.s, o), __shfl_xor_sync(0xFFFFFFFFu, v.e, o)};
            v.add(w);
        }
    }
    __syncthreads();
    return v;
}

__device__ __forceinline__ void chunk_of(int64_t C, int64_t& begin, int64_t& end) {
    const int64_t chunk = (C + gridDim.x - 1) / gridDim.x;
    begin = (int64_t)blockIdx.x * chunk;
    end = begin + chunk < C ? begin + chunk : C;
    if (begin > C) begin = C;
}

// True in every thread of the CTA that arrived last at `ticket`, among
// `ctas` arriving CTAs (the whole grid by default).  The caller's global
// writes are fenced before arriving.
__device__ bool last_to_arrive(uint32_t* ticket, unsigned ctas) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == ctas - 1);
    __syncthreads();
    return last;
}
__device__ bool last_to_arrive(uint32_t* ticket) { return last_to_arrive(ticket, gridDim.x); }

// RN(a / b) for b > 0 from rb = RN(1 / b) with one multiply and two FMAs:
// q0 = RN(a rb) lies within one ulp of a / b, the remainder a - q0 b is then
// exact in an FMA, and one correction step q0 + (a - q0 b) rb rounds to the
// correctly rounded quotient (Markstein's theorem on division with a
// correctly rounded reciprocal, IBM J. Res. Dev. 34(1), 1990).  Zero, tiny
// (|q0| < 2^-960: the remainder near the subnormal range) and non-finite
// quotients take the plain division; the test reads q0's exponent field
// with integer operations, leaving the FP64 pipe to the arithmetic.
__device__ __forceinline__ double div_rn(double a, double b, double rb) {
    const double q0 = a * rb;
    const unsigned ex = (unsigned)((unsigned long long)__double_as_longlong(q0) >> 52) & 0x7FFu;
    if (ex < 1023u - 960u || ex == 0x7FFu) return a / b;
    return fma(fma(-q0, b, a), rb, q0);
}

// Finite test on the exponent bits (integer ALU; the statistics kernel is
// bound by its FP64 pipe).
__device__ __forceinline__ bool finite_bits(double x) {
    return ((unsigned long long)__double_as_longlong(x) & 0x7FF0000000000000ULL) !=
           0x7FF0000000000000ULL;
}

// Mean and sum of squared deviations of one cell's trial estimates
// I_t = V S1_t / n, S1_t = row[t * chunks].x.  With TMAX > 0 (and T <= TMAX)
// the estimates stay in registers between the two passes; with TMAX = 0
// the second pass computes them again (the same bits).
constexpr int kStatsRegTrials = 16;   // the statistics kernels are capped at 80
                                       // registers (3 CTAs per SM): measured faster
                                       // than 126 registers without spills
template <int TMAX>
__device__ __forceinline__ void cell_moments(const double2* row, int64_t chunks, int T, double V,
                                             double n, double rn, double Td, double rT,
                                             double& mean, double& ss, bool& finite) {
    double s = 0.0;
    ss = 0.0;
    if constexpr (TMAX > 0) {
        double x[TMAX];
#pragma unroll
        for (int t = 0; t < TMAX; ++t) {
            if (t < T) {
                const double S1 = row[t * chunks].x;
                finite = finite && finite_bits(S1);
                x[t] = div_rn(V * S1, n, rn);
                s += x[t];
            }
        }
        mean = div_rn(s, Td, rT);
#pragma unroll
        for (int t = 0; t < TMAX; ++t) {
            if (t < T) {
                const double e = x[t] - mean;
                ss = fma(e, e, ss);
            }
        }
    } else {
        for (int t = 0; t < T; ++t) {
            const double S1 = row[t * chunks].x;
            finite = finite && finite_bits(S1);
            s += div_rn(V * S1, n, rn);
        }
        mean = div_rn(s, Td, rT);
        for (int t = 0; t < T; ++t) {
            const double e = div_rn(V * row[t * chunks].x, n, rn) - mean;
            ss = fma(e, e, ss);
        }
    }
}

// How many CTAs of the (fixed) grid take part in a selection step over
// `work` units, at least `per_cta` units each: CTAs beyond that would only
// add block reductions.  A function of the level's size only, so the
// reduction order, and every bit of the result, stays the same on any GPU.
constexpr int64_t kStatsWorkPerCta = 4096;   // (cell, trial) partial sums
constexpr int64_t kCellsPerCta = 1024;       // cells, for flag and compaction
__device__ __forceinline__ int active_ctas(int64_t work, int64_t per_cta) {
    const int64_t g = (work + per_cta - 1) / per_cta;
    return (int)(g < 1 ? 1 : (g < (int64_t)gridDim.x ? g : (int64_t)gridDim.x));
}
// The contiguous chunk of C cells owned by CTA blockIdx.x of G.
__device__ __forceinline__ void chunk_of(int64_t C, int G, int64_t& begin, int64_t& end) {
    const int64_t chunk = (C + G - 1) / G;
    begin = (int64_t)blockIdx.x * chunk;
    end = begin + chunk < C ? begin + chunk : C;
    if (begin > C) begin = C;
}

// Sums of two doubles over the CTA in a fixed order (lane butterfly, then
// the warps in order), returned to every thread.
__device__ double2 block_sum2(double a, double b) {
    __shared__ double2 s[32];
    __shared__ double2 total;
    a = warp_sum(a);
    b = warp_sum(b);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s[warp] = make_double2(a, b);
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 t = make_double2(0.0, 0.0);
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t.x += s[w].x;
            t.y += s[w].y;
        }
        total = t;
    }
    __syncthreads();
    const double2 r = total;
    __syncthreads();
    return r;
}

}  // namespace

// Each step below is a device body run by one grid (or, for a batch of
// integrals, by row blockIdx.y of a 2-D grid) and a thin kernel around it.

// Reset the tree state of a run: level 1 is the full lattice, with its work
// decomposition.
__device__ __forceinline__ void init_state_body(const Desc* __restrict__ desc, State* st,
                                                int64_t level1_cells) {
    uint32_t* w = reinterpret_cast<uint32_t*>(st);
    for (size_t i = threadIdx.x; i < sizeof(State) / 4; i += blockDim.x) w[i] = 0u;
    __syncthreads();
    if (threadIdx.x == 0) {
        st->cells[1] = level1_cells;
        st->uplan[1] = level_plan(*desc, level1_cells);
    }
}

// Step (b1): per cell the mean and sample spread (ddof 1) of the trial
// estimates I_{c,t} = V S1 / n; over the level the mean mu and population
// standard deviation sigma of the spreads; theta = mu + m sigma.  FP64 runs
// at two operations per SM per clock on GB300, so the kernel keeps FP64
// divisions out of its loops: I_{c,t} and the mean are correctly rounded
// quotients from precomputed reciprocals (div_rn; the same bits as a
// division, so a cell whose trials agree has spread 0 exactly), up to 16
// trials' estimates stay in registers between the two passes, and the
// moments of the spreads are taken in two passes with plain sums -- per CTA
// over its cells, then over the CTAs' (count, mean, M2) -- instead of
// pairwise merges.
__device__ __forceinline__ void cell_stats_body(const Desc* __restrict__ desc, State* st,
                                                double2* __restrict__ sums,
                                                double2* __restrict__ cell_stats, double* part,
                                                int level) {
    const Desc& D = *desc;
    const int64_t C = st->cells[level];
    if (C <= 0) return;
    const int T = D.T;
    // The sampling kernel left the level plan's `chunks` partial sums per
    // (cell, trial) tile, contiguous per tile; add them in order and keep the
    // total in the tile's first slot.
    const int64_t chunks = st->uplan[level].chunks;
    const int G = active_ctas(C * T * chunks, kStatsWorkPerCta);
    if ((int)blockIdx.x >= G) return;
    const double V = D.volume[level], n = (double)D.n, Td = (double)T;
    const double rn = 1.0 / n, rT = 1.0 / Td, inv_T1 = 1.0 / (T - 1);
    int64_t begin, end;
    chunk_of(C, G, begin, end);

    bool finite = true;
    double tsum = 0.0;
    int tcount = 0;
    for (int64_t q = begin + threadIdx.x; q < end; q += blockDim.x) {
        if (!in_bounds(st, (q + 1) * T * chunks - 1, cap_partial_sums(D), kSiteSumsRead) ||
            !in_bounds(st, q, D.cap_cells, kSiteStatsWrite))
            continue;
        double2* row = sums + q * T * chunks;
        if (chunks > 1) {
            for (int t = 0; t < T; ++t) {
                double2 S = row[t * chunks];
                for (int64_t c = 1; c < chunks; ++c) {
                    S.x += row[t * chunks + c].x;
                    S.y += row[t * chunks + c].y;
                }
                row[t * chunks] = S;
            }
        }
        // Only S1 enters the method; S2 (a within-cell diagnostic) may
        // overflow in the FP32 modes when |f| exceeds ~1.8e19.
        double mean, ss;
        if (T <= kStatsRegTrials)
            cell_moments<kStatsRegTrials>(row, chunks, T, V, n, rn, Td, rT, mean, ss, finite);
        else
            cell_moments<0>(row, chunks, T, V, n, rn, Td, rT, mean, ss, finite);
        const double spread = sqrt(ss * inv_T1);
        cell_stats[q] = make_double2(mean, spread);
        tsum += spread;
        ++tcount;
    }
    if (!finite) atomicMax(&st->status, ZMC_ERR_NONFINITE);
    // this CTA's count, mean and M2 of its spreads (the second pass reads
    // back what this thread wrote)
    const double2 sc = block_sum2(tsum, (double)tcount);
    const double cmean = sc.y > 0.0 ? sc.x / sc.y : 0.0;
    double m2 = 0.0;
    for (int64_t q = begin + threadIdx.x; q < end; q += blockDim.x) {
        if (!in_bounds(st, (q + 1) * T * chunks - 1, cap_partial_sums(D), kSiteSumsRead) ||
            !in_bounds(st, q, D.cap_cells, kSiteStatsWrite))
            continue;
        const double e = cell_stats[q].y - cmean;
        m2 = fma(e, e, m2);
    }
    const double m2c = block_sum2(m2, 0.0).x;
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 0] = sc.y;
        part[3 * blockIdx.x + 1] = cmean;
        part[3 * blockIdx.x + 2] = m2c;
    }
    if (!last_to_arrive(&st->ticket[0], G)) return;

    // The level's moments from the CTAs': mu = sum n_b mean_b / N and
    // M2 = sum (M2_b + n_b (mean_b - mu)^2).
    double a = 0.0, nn = 0.0;
    for (int b = threadIdx.x; b < G; b += blockDim.x) {
        const double nb = __ldcg(part + 3 * b);
        a += nb * __ldcg(part + 3 * b + 1);
        nn += nb;
    }
    const double2 an = block_sum2(a, nn);
    const double mu = an.y > 0.0 ? an.x / an.y : 0.0;
    double m2g = 0.0;
    for (int b = threadIdx.x; b < G; b += blockDim.x) {
        const double nb = __ldcg(part + 3 * b);
        const double e = __ldcg(part + 3 * b + 1) - mu;
        m2g += __ldcg(part + 3 * b + 2) + nb * e * e;
    }
    m2g = block_sum2(m2g, 0.0).x;
    if (threadIdx.x == 0) {
        const double sigma = an.y > 0.0 ? sqrt(m2g / an.y) : 0.0;
        st->mu[level] = mu;
        st->sigma[level] = sigma;
        st->theta[level] = mu + D.m * sigma;
        st->ticket[0] = 0u;
    }
}

// Step (b2): flag cells whose spread is strictly larger than theta (never at
// the last level), count them per CTA, and let the last CTA scan the counts,
// apply the refinement budget and publish the next level's size.
__device__ __forceinline__ void flag_count_body(const Desc* __restrict__ desc, State* st,
                                                const double2* __restrict__ cell_stats,
                                                int64_t* part_count, int64_t* part_offset,
                                                double* part_margin, int level) {
    const Desc& D = *desc;
    const int64_t C = st->cells[level];
    if (C <= 0) return;
    const double theta = st->theta[level];
    const bool can_flag = level < D.depth;
    const int G = active_ctas(C, kCellsPerCta);
    if ((int)blockIdx.x >= G) return;
    int64_t begin, end;
    chunk_of(C, G, begin, end);

    // The margin min |s - theta| / theta: a correctly rounded division by
    // theta > 0 is monotone, so the CTAs keep min |s - theta| and the last
    // one divides once, which gives the same bits as the minimum of the
    // quotients.
    int64_t cnt = 0;
    double mm = INFINITY;
    for (int64_t q = begin + threadIdx.x; q < end; q += blockDim.x) {
        if (!in_bounds(st, q, D.cap_cells, kSiteStatsRead)) continue;
        const double s = cell_stats[q].y;
        cnt += (can_flag && s > theta) ? 1 : 0;
        mm = fmin(mm, fabs(s - theta));
    }
    __shared__ int64_t s_cnt[32];
    __shared__ double s_mm[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
        mm = fmin(mm, __shfl_xor_sync(0xFFFFFFFFu, mm, o));
    }
    if (lane == 0) { s_cnt[warp] = cnt; s_mm[warp] = mm; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t c = 0;
        double m = INFINITY;
        for (int w = 0; w < nw; ++w) { c += s_cnt[w]; m = fmin(m, s_mm[w]); }
        part_count[blockIdx.x] = c;
        part_margin[blockIdx.x] = m;
    }
    if (!last_to_arrive(&st->ticket[1], G)) return;

    // Exclusive scan of the per-CTA counts over the whole CTA: thread j takes
    // a run of `per` consecutive CTAs' counts, the runs' totals are scanned
    // across the warps, and each thread then writes its run's offsets.
    const int per = (G + (int)blockDim.x - 1) / (int)blockDim.x;
    const int b0 = min(G, (int)threadIdx.x * per), b1 = min(G, b0 + per);
    int64_t mine = 0;
    double mloc = INFINITY;
    for (int b = b0; b < b1; ++b) {
        mine += __ldcg(part_count + b);
        mloc = fmin(mloc, __ldcg(part_margin + b));
    }
    int64_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
        mloc = fmin(mloc, __shfl_xor_sync(0xFFFFFFFFu, mloc, o));
    }
    if (lane == 31) s_cnt[warp] = incl;
    if (lane == 0) s_mm[warp] = mloc;
    __syncthreads();
    int64_t before = 0, run = 0;
    double m = INFINITY;
    for (int w = 0; w < nw; ++w) {
        if (w < warp) before += s_cnt[w];
        run += s_cnt[w];
        m = fmin(m, s_mm[w]);
    }
    int64_t off = before + incl - mine;
    for (int b = b0; b < b1; ++b) {
        part_offset[b] = off;
        off += __ldcg(part_count + b);
    }
    if (threadIdx.x == 0) {
        const int64_t F = run;
        const int64_t per_cell = D.n * (int64_t)D.T;
        const int64_t samples = st->samples + C * per_cell;
        st->samples = samples;
        int refine = 0;
        int64_t flagged = F;
        if (F > 0) {
            const uint64_t next = (uint64_t)F * (uint64_t)D.K;
            const int64_t room = (D.max_samples - samples) / per_cell;
            if (next > (uint64_t)D.max_cells || next > (uint64_t)room ||
                next > (uint64_t)D.cap_cells) {
                atomicMax(&st->status, ZMC_ERR_BUDGET);
                flagged = 0;
            } else {
                refine = 1;
                st->cells[level + 1] = (int64_t)next;
                st->uplan[level + 1] = level_plan(D, (int64_t)next);
            }
        }
        st->flagged[level] = flagged;
        st->refine[level] = refine;
        st->min_margin[level] =
            (can_flag && theta > 0.0 && m < INFINITY) ? m / theta : INFINITY;
        st->levels_run = level;
        st->ticket[1] = 0u;
    }
}

// Step (b3): write the coordinates of the flagged cells, in slot order, as
// the next level's parent list (the children themselves are implicit:
// child slot r*K + digit); add the accepted cells' mean and spread^2 / T to
// this level's compensated partial sums.
__device__ __forceinline__ void compact_body(const Desc* __restrict__ desc, State* st,
                                             const double2* __restrict__ cell_stats,
                                             const int64_t* __restrict__ part_offset,
                                             const uint32_t* __restrict__ parents_prev,
                                             uint32_t* __restrict__ parents_next,
                                             double* __restrict__ part_acc, int level) {
    const Desc& D = *desc;
    const int64_t C = st->cells[level];
    if (C <= 0) return;
    const bool refine = st->refine[level] != 0;
    const double theta = st->theta[level];
    const int d = D.d;
    const int G = active_ctas(C, kCellsPerCta);
    if ((int)blockIdx.x >= G) return;
    int64_t begin, end;
    chunk_of(C, G, begin, end);

    __shared__ int s_warp[32];
    __shared__ int s_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t offset = refine ? part_offset[blockIdx.x] : 0;
    CSum val{0.0, 0.0}, var{0.0, 0.0};
    for (int64_t q0 = begin; q0 < end; q0 += blockDim.x) {
        const int64_t q = q0 + threadIdx.x;
        const bool valid = q < end && in_bounds(st, q, D.cap_cells, kSiteStatsRead);
        double2 ms = valid ? cell_stats[q] : make_double2(0.0, 0.0);
        const bool flag = valid && refine && ms.y > theta;
        const unsigned ballot = __ballot_sync(0xFFFFFFFFu, flag);
        const int rank_in_warp = __popc(ballot & ((1u << lane) - 1u));
        if (lane == 0) s_warp[warp] = __popc(ballot);
        __syncthreads();
        if (threadIdx.x == 0) {
            int run = 0;
            for (int w = 0; w < nw; ++w) { const int c = s_warp[w]; s_warp[w] = run; run += c; }
            s_total = run;
        }
        __syncthreads();
        if (flag) {
            const int64_t r = offset + s_warp[warp] + rank_in_warp;
            if (in_bounds(st, r * d + d - 1, cap_parents(D), kSiteParentWrite))
                for (int i = 0; i < d; ++i)
                    parents_next[r * d + i] =
                        (uint32_t)cell_coord(D, level, q, i, parents_prev, st);
        } else if (valid) {
            val.add(ms.x);
            var.add(ms.y * ms.y);  // divided by T once, in the final reduction
        }
        offset += s_total;
        __syncthreads();
    }
    val = block_csum(val);
    var = block_csum(var);
    if (threadIdx.x == 0) {
        double* p = part_acc + (size_t)blockIdx.x * 4;
        p[0] = val.s; p[1] = val.e; p[2] = var.s; p[3] = var.e;
    }
    if (!last_to_arrive(&st->ticket[2], G)) return;

    // the level's slot: the CTAs' compensated partials added in CTA order
    CSum lv{0.0, 0.0}, lw{0.0, 0.0};
    for (int b = threadIdx.x; b < G; b += blockDim.x) {
        const double* p = part_acc + (size_t)b * 4;
        lv.add(CSum{__ldcg(p), __ldcg(p + 1)});
        lw.add(CSum{__ldcg(p + 2), __ldcg(p + 3)});
    }
    lv = block_csum(lv);
    lw = block_csum(lw);
    if (threadIdx.x == 0) {
        double* p = part_acc + ((size_t)kSelGrid + level) * 4;
        p[0] = lv.s; p[1] = lv.e; p[2] = lw.s; p[3] = lw.e;
        st->ticket[2] = 0u;
    }
}

// Step (c): the compensated sum of every level's accepted partial sums, and
// the result record.  One CTA.
__device__ __forceinline__ void final_body(const Desc* __restrict__ desc,
                                           const State* __restrict__ st,
                                           const double* __restrict__ part_acc,
                                           zmc_result* __restrict__ out) {
    const int levels = st->levels_run;
    CSum val{0.0, 0.0}, var{0.0, 0.0};
    for (int L = 1 + threadIdx.x; L <= levels; L += blockDim.x) {
        const double* p = part_acc + ((size_t)kSelGrid + L) * 4;
        val.add(CSum{p[0], p[1]});
        var.add(CSum{p[2], p[3]});
    }
    val = block_csum(val);
    var = block_csum(var);
    if (threadIdx.x == 0) {
        out->value = val.s + val.e;
        out->std = sqrt((var.s + var.e) / desc->T);
        int64_t cells = 0;
        for (int L = 1; L <= ZMC_MAX_DEPTH; ++L) {
            const bool ran = L <= levels;
            out->cells_per_level[L - 1] = ran ? st->cells[L] : 0;
            out->flagged_per_level[L - 1] = ran ? st->flagged[L] : 0;
            out->theta_per_level[L - 1] = ran ? st->theta[L] : 0.0;
            out->mu_per_level[L - 1] = ran ? st->mu[L] : 0.0;
            out->sigma_per_level[L - 1] = ran ? st->sigma[L] : 0.0;
            out->min_margin_per_level[L - 1] = ran ? st->min_margin[L] : 0.0;
            if (ran) cells += st->cells[L];
        }
        out->cells_evaluated = cells;
        out->samples = st->samples;
        out->levels_run = levels;
        out->status = st->status;
    }
}

// ---------------------------------------------------------------- kernels
// One integration: the buffers are kernel arguments.
__global__ void zmc_init_state(const Desc* desc, State* st, int64_t level1_cells) {
    init_state_body(desc, st, level1_cells);
}
__global__ void __launch_bounds__(kSelThreads, 3)
zmc_cell_stats(const Desc* desc, State* st, double2* sums, double2* cell_stats, double* part,
               int level) {
    cell_stats_body(desc, st, sums, cell_stats, part, level);
}
__global__ void __launch_bounds__(kSelThreads)
zmc_flag_count(const Desc* desc, State* st, const double2* cell_stats, int64_t* part_count,
               int64_t* part_offset, double* part_margin, int level) {
    flag_count_body(desc, st, cell_stats, part_count, part_offset, part_margin, level);
}
__global__ void __launch_bounds__(kSelThreads)
zmc_compact(const Desc* desc, State* st, const double2* cell_stats,
            const int64_t* part_offset, const uint32_t* parents_prev, uint32_t* parents_next,
            double* part_acc, int level) {
    compact_body(desc, st, cell_stats, part_offset, parents_prev, parents_next, part_acc, level);
}
__global__ void __launch_bounds__(kSelThreads)
zmc_final(const Desc* desc, const State* st, const double* part_acc, zmc_result* out) {
    final_body(desc, st, part_acc, out);
}

// A batch of integrations: row blockIdx.y of the grid works on items[y].
// Level L reads the parent list written by level L-1 (ping-pong by parity).
__global__ void zmc_init_state_batch(const Buffers* items, const int64_t* level1_cells) {
    init_state_body(items[blockIdx.y].desc, items[blockIdx.y].state, level1_cells[blockIdx.y]);
}
__global__ void __launch_bounds__(kSelThreads, 3)
zmc_cell_stats_batch(const Buffers* items, int level) {
    const Buffers& b = items[blockIdx.y];
    cell_stats_body(b.desc, b.state, b.sums, b.cell_stats, b.part_stats, level);
}
__global__ void __launch_bounds__(kSelThreads)
zmc_flag_count_batch(const Buffers* items, int level) {
    const Buffers& b = items[blockIdx.y];
    flag_count_body(b.desc, b.state, b.cell_stats, b.part_count, b.part_offset, b.part_margin,
                    level);
}
__global__ void __launch_bounds__(kSelThreads)
zmc_compact_batch(const Buffers* items, int level) {
    const Buffers& b = items[blockIdx.y];
    compact_body(b.desc, b.state, b.cell_stats, b.part_offset, b.parents[level & 1],
                 b.parents[(level + 1) & 1], b.part_acc, level);
}
__global__ void __launch_bounds__(kSelThreads)
zmc_final_batch(const Buffers* items, zmc_result* out) {
    const Buffers& b = items[blockIdx.y];
    final_body(b.desc, b.state, b.part_acc, &out[blockIdx.y]);
}

// Philox words for bit-exact checks of the generator used by kernel (a).
// Same code path as the sampling kernel: (c1, c2, c3) play (t, q, L).
__global__ void zmc_philox_fill(const PhiloxKeys keys, uint32_t c0, uint32_t c1, uint32_t c2,
                                uint32_t c3, int64_t count, uint4* out) {
    const StreamConst sc = stream_const(keys, c1, c2, c3);
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < count;
         b += (int64_t)gridDim.x * blockDim.x)
        out[b] = philox_stream(keys, sc, c0 + (uint32_t)b);
}

// The uniforms of points [first, first + count) of one (level, slot, trial)
// stream, all d dimensions, as the sampling kernel forms them (1.m values
// from philox_stream with the word and field layout of the sampling loop),
// minus the exact shift.
__global__ void zmc_uniforms_fill(const PhiloxKeys keys, uint32_t level, uint32_t slot,
                                  uint32_t trial, int d, int mode, int64_t first, int64_t count,
                                  double* out) {
    const StreamConst sc = stream_const(keys, trial, slot, level);
    const int G = points_per_group(mode), B = blocks_per_group(mode);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count * d;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = first + e / d;
        const int i = (int)(e % d);
        const uint32_t c0 = (uint32_t)(((s / G) * d + i) * B);
        const uint4 w = philox_stream(keys, sc, c0);
        const int lane = (int)(s % G);
        double u;
        if (mode == ZMC_FP64) {
            const uint32_t word = lane == 0 ? w.x : lane == 1 ? w.y : lane == 2 ? w.z : w.w;
            u = one_plus_word_f64(word) - (1.0 - 0x1p-33);
        } else {
            const uint4 w2 = philox_stream(keys, sc, c0 + 1);
            float v[11];
            fields_1m(w, v[0], v[1], v[2], v[3], v[4]);
            fields_1m(w2, v[5], v[6], v[7], v[8], v[9]);
            v[10] = cross_1m(w, w2);
            u = (double)(v[lane] - (1.0f - 0x1p-24f));
        }
        out[e] = u;
    }
}

cudaError_t launch_uniforms(uint64_t seed, int level, uint32_t slot, uint32_t trial, int d,
                            int mode, int64_t first, int64_t count, double* out, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    int64_t blocks = (count * d + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    zmc_uniforms_fill<<<(int)blocks, 256, 0, s>>>(philox_keys(seed), (uint32_t)level, slot,
                                                  trial, d, mode, first, count, out);
    return cudaGetLastError();
}

PhiloxKeys philox_keys(uint64_t seed) {
    PhiloxKeys K;
    uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu), k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        K.k0[r] = k0;
        K.k1[r] = k1;
        k0 += kPhiloxWeylA;
        k1 += kPhiloxWeylB;
    }
    return K;
}

// ------------------------------------------------------------- launchers

cudaError_t launch_init(const Buffers& b, int64_t level1_cells, cudaStream_t s) {
    zmc_init_state<<<1, 256, 0, s>>>(b.desc, b.state, level1_cells);
    return cudaGetLastError();
}

cudaError_t launch_select(const Buffers& b, int level, const uint32_t* parents_prev,
                          uint32_t* parents_next, cudaStream_t s) {
    zmc_cell_stats<<<kSelGrid, kSelThreads, 0, s>>>(b.desc, b.state, b.sums, b.cell_stats,
                                                    b.part_stats, level);
    zmc_flag_count<<<kSelGrid, kSelThreads, 0, s>>>(b.desc, b.state, b.cell_stats,
                                                    b.part_count, b.part_offset,
                                                    b.part_margin, level);
    zmc_compact<<<kSelGrid, kSelThreads, 0, s>>>(b.desc, b.state, b.cell_stats, b.part_offset,
                                                 parents_prev, parents_next, b.part_acc, level);
    return cudaGetLastError();
}

cudaError_t launch_final(const Buffers& b, cudaStream_t s) {
    zmc_final<<<1, kSelThreads, 0, s>>>(b.desc, b.state, b.part_acc, b.result);
    return cudaGetLastError();
}

cudaError_t launch_init_batch(const Buffers* items, const int64_t* level1_cells, int count,
                              cudaStream_t s) {
    zmc_init_state_batch<<<dim3(1, count), 256, 0, s>>>(items, level1_cells);
    return cudaGetLastError();
}

cudaError_t launch_select_batch(const Buffers* items, int count, int level, cudaStream_t s) {
    const dim3 grid(kSelGrid, count);
    zmc_cell_stats_batch<<<grid, kSelThreads, 0, s>>>(items, level);
    zmc_flag_count_batch<<<grid, kSelThreads, 0, s>>>(items, level);
    zmc_compact_batch<<<grid, kSelThreads, 0, s>>>(items, level);
    return cudaGetLastError();
}

cudaError_t launch_final_batch(const Buffers* items, zmc_result* out, int count, cudaStream_t s) {
    zmc_final_batch<<<dim3(1, count), kSelThreads, 0, s>>>(items, out);
    return cudaGetLastError();
}

// ------------------------------------------------ no-allocation variant
// zmc_level_stats_noalloc: the per-cell statistics and level threshold of
// zmc_cell_stats for per-(cell, trial) sums the caller already holds, with
// all scratch in the static array below instead of library-allocated
// buffers.  One CTA per kNoAllocCellsPerBlock cells, so the array bounds the
// number of cells a call accepts.
constexpr int kNoAllocCellsPerBlock = 1024;
constexpr int kNoAllocMaxBlocks = 1024;
constexpr int64_t kNoAllocMaxCells = (int64_t)kNoAllocCellsPerBlock * kNoAllocMaxBlocks;

// Per-CTA (count, mean, M2) partials, then the arrival ticket.  24 KiB +
// 256 B, held by every GPU that loads the library until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxBlocks * 3 + 32];

__global__ void __launch_bounds__(kSelThreads)
zmc_level_stats_noalloc_kernel(const double2* __restrict__ sums, int64_t C, int T, double n,
                               double V, double m, double2* __restrict__ cell_stats,
                               double* __restrict__ level_stats, double* scratch) {
    double* part = scratch;
    uint32_t* ticket = reinterpret_cast<uint32_t*>(scratch + kNoAllocMaxBlocks * 3);
    int64_t begin, end;
    chunk_of(C, begin, end);
    Moments acc{0.0, 0.0, 0.0};
    for (int64_t q = begin + threadIdx.x; q < end; q += blockDim.x) {
        const double2* row = sums + q * T;
        double s = 0.0;
        for (int t = 0; t < T; ++t) s += V * row[t].x / n;
        const double mean = s / T;
        double ss = 0.0;
        for (int t = 0; t < T; ++t) {
            const double e = V * row[t].x / n - mean;
            ss += e * e;
        }
        const double spread = sqrt(ss / (T - 1));
        cell_stats[q] = make_double2(mean, spread);
        acc = merge(acc, Moments{1.0, spread, 0.0});
    }
    acc = block_merge(acc);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 0] = acc.n;
        part[3 * blockIdx.x + 1] = acc.mean;
        part[3 * blockIdx.x + 2] = acc.m2;
    }
    if (!last_to_arrive(ticket)) return;
    Moments all{0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
        all = merge(all, Moments{__ldcg(part + 3 * b), __ldcg(part + 3 * b + 1),
                                 __ldcg(part + 3 * b + 2)});
    all = block_merge(all);
    if (threadIdx.x == 0) {
        const double sigma = sqrt(all.m2 / all.n);
        level_stats[0] = all.mean;
        level_stats[1] = sigma;
        level_stats[2] = all.mean + m * sigma;
        *ticket = 0u;
    }
}

namespace {
// The device address of the scratch array on the current device (in host
// code its name is only a host-side stand-in).  Looked up on every call, with
// the caller's device current: the lookup allocates nothing, and a cached
// address would go stale if the caller reset the device's context.
int noalloc_scratch(double** out, std::string* why) {
    double* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
        *why = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return ZMC_ERR_CUDA;
    }
    *out = p;
    return ZMC_OK;
}

thread_local std::string g_noalloc_error;
}  // namespace

const char* noalloc_last_error() { return g_noalloc_error.c_str(); }

int level_stats_noalloc(const double* sums, int64_t cells, int trials, int64_t n, double volume,
                        double sigma_multiplier, double* cell_stats, double* level_stats,
                        cudaStream_t s) {
    if (!sums || !cell_stats || !level_stats) {
        g_noalloc_error = "sums, cell_stats and level_stats must be device pointers";
        return ZMC_ERR_ARG;
    }
    if (cells < 1 || cells > kNoAllocMaxCells) {
        g_noalloc_error = "cells must be in 1.." + std::to_string(kNoAllocMaxCells) +
                          " (the size of the static scratch of this entry point)";
        return ZMC_ERR_ARG;
    }
    if (trials < 2 || n < 1 || !isfinite(volume) || !isfinite(sigma_multiplier) ||
        sigma_multiplier < 0.0) {
        g_noalloc_error = "need trials >= 2, n >= 1, finite volume, finite sigma_multiplier >= 0";
        return ZMC_ERR_ARG;
    }
    double* scratch = nullptr;
    if (int rc = noalloc_scratch(&scratch, &g_noalloc_error)) return rc;
    // The scratch keeps the previous call's contents: the ticket must start at 0.
    cudaError_t e = cudaMemsetAsync(scratch + kNoAllocMaxBlocks * 3, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) {
        const int grid = (int)((cells + kNoAllocCellsPerBlock - 1) / kNoAllocCellsPerBlock);
        zmc_level_stats_noalloc_kernel<<<grid, kSelThreads, 0, s>>>(
            reinterpret_cast<const double2*>(sums), cells, trials, (double)n, volume,
            sigma_multiplier, reinterpret_cast<double2*>(cell_stats), level_stats, scratch);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        g_noalloc_error = std::string("launch: ") + cudaGetErrorString(e);
        return ZMC_ERR_CUDA;
    }
    return ZMC_OK;
}

cudaError_t launch_philox(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                          uint32_t c3, int64_t count, uint32_t* out, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    int64_t blocks = (count + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    zmc_philox_fill<<<(int)blocks, 256, 0, s>>>(philox_keys(seed), c0, c1, c2, c3, count,
                                               reinterpret_cast<uint4*>(out));
    return cudaGetLastError();
}

}  // namespace zmc
