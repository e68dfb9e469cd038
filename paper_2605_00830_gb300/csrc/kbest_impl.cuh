// kbest_impl.cuh -- sm_103a K-Best kernels (templates; instantiated per edge-label plane
// count in kbest_b0.cu, kbest_b2.cu and kbest_b8.cu; the S0 packing kernel and the dispatch
// live in kbest_kernels.cu).
//
//   kbest_kernel          S1-S5 for every pair of a size class: persistent one-CTA teams pull
//                         pairs from a device work queue; per level they build per-node
//                         neighbour bitsets, score every successor with AND/XOR + popcount
//                         against the staged vertex-cost row, select the best K exactly
//                         (a PED histogram, a stable compaction and a counting placement),
//                         write the kept children in key order and stage the next cost row;
//                         finally they complete the leaves and take the argmin.
//   kbest_cluster_kernel  the same with a team of 2-16 CTAs in a thread-block cluster, for
//                         classes with fewer pairs than SMs and large pairs or beams.
//
// Method: Algorithm 1 of Dabah & Herten (branching Sec. 4.1.1, evaluation Sec. 4.1.2 and
// Algorithm 2, selection Sec. 4.2, leaf insertions Sec. 4.4). The paper's GPU design
// (one block per node, a lambda walk per successor, atomic top-L lists) is replaced here:
// the implied edge cost of substituting v_i by u is computed from bitsets,
//     P     = images of the already-substituted g1 neighbours of v_i,
//     Img   = images of every substituted g1 vertex,
//     A2[u] = neighbours of u in g2,
//   inserted edges   = popc(A2[u] & Img & ~P)
//   deleted edges    = popc(P & ~A2[u]) + (# g1 neighbours of v_i that were deleted)
//   relabelled edges = popc(A2[u] & P & OR_b(PL_b ^ L2_b[u]))
// and when insertion and deletion cost the same, the first two fold into one
// popc((A2[u] & Img) ^ P) since P is a subset of Img.
#pragma once
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "fastged_internal.h"

namespace fastged {

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int warp_sum(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// bits k of word w with k < i
__device__ __forceinline__ uint64_t low_mask(int i, int w)
{
    const int lo = w * 64;
    if (i >= lo + 64) return ~0ull;
    if (i <= lo) return 0ull;
    return (1ull << (i - lo)) - 1ull;
}

// ------------------------------------------------------------------------------------
// K-Best teams
// ------------------------------------------------------------------------------------
// Team scalars: in shared memory for a one-CTA team, in the cluster's global scratch for a
// cluster team (MW = warps the team may have).
template <int MW>
struct TeamSharedT {
    int pair;
    int cnt;
    int mx;
    int wmin[MW];  // least successor PED each warp scored at this level
    int wn[MW];    // successors each warp scored at this level
    int wlt[MW];
    int weq[MW];
    unsigned long long wbest[MW];
};
using TeamShared = TeamSharedT<kMaxWarps>;
using TeamSharedCl = TeamSharedT<kMaxClusterWarps>;

__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned cluster_size()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

// Barrier over every thread of the cluster; writes before it (shared or global) are visible
// to every thread of the cluster after it (release / acquire at cluster scope).
__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
                 ::: "memory");
}

// The threads solving one pair: one CTA, or every CTA of a cluster (CL).
template <bool CL>
struct Team {
    int tid, T, warp, NW;
    __device__ __forceinline__ Team()
    {
        if (CL) {
            tid = (int)cluster_rank() * (int)blockDim.x + (int)threadIdx.x;
            T = (int)cluster_size() * (int)blockDim.x;
        } else {
            tid = (int)threadIdx.x;
            T = (int)blockDim.x;
        }
        warp = tid >> 5;
        NW = T >> 5;
    }
    __device__ __forceinline__ void sync() const
    {
        if (CL) cluster_barrier();
        else __syncthreads();
    }
};

template <typename Word>
struct Regions {
    int32_t *hist, *alpha2, *crow, *sbase, *sel, *selped, *klist, *kped, *noff, *nbr, *cand;
    int32_t *ped0, *ped1;
    Word *a2t, *l2t, *img0, *img1, *P, *PL, *imgl;
    uint8_t *map0, *map1;
};

// A kept child is stored in the selection list as (parent slot << 11) | j, j = 0..n2.
constexpr int kSelShift = 11;

__device__ __forceinline__ int popcw(uint32_t x) { return __popc(x); }
__device__ __forceinline__ int popcw(uint64_t x) { return __popcll(x); }

#ifdef FASTGED_PHASE_TIMERS
// profiling builds only: cycles thread 0 of every team spends in each phase
#define PHASE_MARK(k)                                        \
    do {                                                     \
        if (threadIdx.x == 0) {                              \
            const long long t_ = clock64();                  \
            ph[k] += t_ - ph_last;                           \
            ph_last = t_;                                    \
        }                                                    \
    } while (0)
#else
#define PHASE_MARK(k) do { } while (0)
#endif

// Lanes of the warp whose 5-bit value equals `v`, among the lanes in `valid`, given the
// ballots b[k] of bit k of every lane's value.
__device__ __forceinline__ unsigned same_value_lanes(unsigned valid, const unsigned b[5], int v)
{
    unsigned m = valid;
#pragma unroll
    for (int k = 0; k < 5; ++k) m &= ((v >> k) & 1) ? b[k] : ~b[k];
    return m;
}

// PED of successor entry k: a packed 32-bit entry (PED << 16 | parent slot << jbits | j) or
// an unpacked 64-bit one (PED << 32 | parent slot << kSelShift | j).
__device__ __forceinline__ int entry_ped(const KParams &p, const int32_t *cand, int64_t k, bool pk)
{
    return pk ? (int)(FG_AT((const uint32_t *)cand, k, FG_N(uint32_t, p.lay.rsize[RG_CAND])) >> 16)
              : (int)(FG_AT((const uint64_t *)cand, k, FG_N(uint64_t, p.lay.rsize[RG_CAND])) >> 32);
}

// Stable compaction of the kept successors of this warp, in enumeration order: every
// candidate with PED < T, and the first q with PED == T counted over the whole team.
// keep_before / eq_before: kept / tied candidates of the warps before this one.
template <typename Word>
__device__ __forceinline__ int compact_kept(const KParams &p, const Regions<Word> &R, int base,
                                           int n, int T, int q, int keep_before, int eq_before,
                                           bool pk)
{
    const int lane = threadIdx.x & 31;
    const int keep0 = keep_before;

    // four chunks of 32 per step: their loads and threshold ballots are independent, so only
    // chunks holding a kept candidate pay for the ordered part
    for (int kb = 0; kb < n; kb += 128) {
        int v[4];
        unsigned le[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = kb + 32 * u + lane;
            v[u] = k < n ? entry_ped(p, R.cand, (int64_t)base + k, pk) : INT_MAX;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) le[u] = __ballot_sync(0xffffffffu, v[u] <= T);
        if ((le[0] | le[1] | le[2] | le[3]) == 0u) continue;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (le[u] == 0u) continue;
            const bool is_eq = (v[u] == T);
            const unsigned eqb = __ballot_sync(0xffffffffu, is_eq);
            const int eq_rank = eq_before + __popc(eqb & lanemask_lt());
            const bool keep = (v[u] < T) || (is_eq && eq_rank < q);
            const unsigned kbm = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int pos = keep_before + __popc(kbm & lanemask_lt());
                FG_AT(R.klist, pos, FG_N(int32_t, p.lay.rsize[RG_KLIST])) = base + kb + 32 * u + lane;
                FG_AT(R.kped, pos, FG_N(int32_t, p.lay.rsize[RG_KPED])) = v[u];
            }
            keep_before += __popc(kbm);
            eq_before += __popc(eqb);
        }
    }
    return keep_before - keep0;
}

// Exact selection used when the kept set reaches past the histogram window: the K-th
// smallest PED is found by bisection over team-wide counts, the kept candidates are
// compacted stably, and ranked by (PED, enumeration order); sel receives successor indices.
template <typename MapT, typename Word, bool CL, typename TS>
__device__ __noinline__ void select_exact(const KParams &p, int32_t *cand, int32_t *klist,
                                          int32_t *kped, int32_t *sel, int32_t *selped, TS &S,
                                          int L, int stride, int newL, int lo, bool pk)
{
    const Team<CL> tm;
    const int tid = tm.tid, lane = threadIdx.x & 31, warp = tm.warp;
    const int T = tm.T, NW = tm.NW;
    const int s_lo = (warp * L) / NW;
#define NKP FG_N(int32_t, p.lay.rsize[RG_KPED])
#define NKL FG_N(int32_t, p.lay.rsize[RG_KLIST])
#define NSE FG_N(int32_t, p.lay.rsize[RG_SEL])
#define NSP FG_N(int32_t, p.lay.rsize[RG_SELPED])
#define NSW ((int64_t)(sizeof(S.wn) / sizeof(S.wn[0])))
    const int base = s_lo * stride, n = FG_AT(S.wn, warp, NSW);
    Regions<Word> R;
    R.cand = cand;
    R.klist = klist;
    R.kped = kped;

    int mx = 0;
    for (int k = lane; k < n; k += 32) mx = max(mx, entry_ped(p, cand, base + k, pk));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (tid == 0) S.mx = 0;
    tm.sync();
    if (lane == 0) atomicMax(&S.mx, mx);
    tm.sync();
    int hi = S.mx;
    if (lo > hi) lo = hi;
    // invariant: count(PED < lo) < newL <= count(PED <= hi)
    while (lo < hi) {
        const int mid = lo + (hi - lo) / 2;
        int cnt = 0;
        for (int k = lane; k < n; k += 32) cnt += (entry_ped(p, cand, base + k, pk) <= mid);
        cnt = warp_sum(cnt);
        tm.sync();
        if (tid == 0) S.cnt = 0;
        tm.sync();
        if (lane == 0) atomicAdd(&S.cnt, cnt);
        tm.sync();
        if (S.cnt >= newL) hi = mid; else lo = mid + 1;
    }
    const int thr = lo;
    int nlt = 0, neq = 0;
    for (int k = lane; k < n; k += 32) {
        const int v = entry_ped(p, cand, base + k, pk);
        nlt += (v < thr);
        neq += (v == thr);
    }
    nlt = warp_sum(nlt);
    neq = warp_sum(neq);
    if (lane == 0) { FG_AT(S.wlt, warp, NSW) = nlt; FG_AT(S.weq, warp, NSW) = neq; }
    tm.sync();
    // the warps' counts are read by all lanes at once (for a cluster team they live in
    // global scratch, so a serial walk would pay one round trip per warp)
    int lt_all = 0, keep_before = 0, eq_before = 0;
    for (int w = lane; w < NW; w += 32) {
        const int lt = FG_AT(S.wlt, w, NSW);
        lt_all += lt;
        if (w < warp) {
            keep_before += lt;
            eq_before += FG_AT(S.weq, w, NSW);
        }
    }
    lt_all = warp_sum(lt_all);
    keep_before = warp_sum(keep_before);
    eq_before = warp_sum(eq_before);
    const int q = newL - lt_all;
    keep_before += min(q, eq_before);
    compact_kept<Word>(p, R, base, n, thr, q, keep_before, eq_before, pk);
    tm.sync();
    // order by (PED, enumeration order); klist is in enumeration order and its entries are
    // increasing, so (kped, klist) is that key
    if (newL <= 2048) {
        for (int a = tid; a < newL; a += T) {
            const int pa = FG_AT(kped, a, NKP);
            int rank = 0;
            for (int b = 0; b < newL; ++b) {
                const int pb = FG_AT(kped, b, NKP);
                rank += (pb < pa) || (pb == pa && b < a);
            }
            // successor index; the caller turns it into (slot, j)
            FG_AT(sel, rank, NSE) = FG_AT(klist, a, NKL);
            FG_AT(selped, rank, NSP) = pa;
        }
        return;
    }
    // large beams: bitonic sort of (kped, klist) in place. Every comparator puts the smaller
    // key at the lower index (each merge starts with a reversed-partner stage), so entries
    // past newL act as +infinity padding up to the next power of two and are never touched.
    int N = 1;
    while (N < newL) N <<= 1;
    auto cmpswap = [&](int i, int j) {
        if (j >= newL) return;
        const int pi = FG_AT(kped, i, NKP), pj = FG_AT(kped, j, NKP);
        const int li = FG_AT(klist, i, NKL), lj = FG_AT(klist, j, NKL);
        if (pj < pi || (pj == pi && lj < li)) {
            FG_AT(kped, i, NKP) = pj;
            FG_AT(kped, j, NKP) = pi;
            FG_AT(klist, i, NKL) = lj;
            FG_AT(klist, j, NKL) = li;
        }
    };
    for (int size = 2; size <= N; size <<= 1) {
        const int half = size >> 1;
        for (int t = tid; t < N / 2; t += T) {
            const int blk = t / half, off = t - blk * half;
            cmpswap(blk * size + off, blk * size + size - 1 - off);
        }
        tm.sync();
        for (int stride = half >> 1; stride > 0; stride >>= 1) {
            for (int t = tid; t < N / 2; t += T) {
                const int blk = t / stride, off = t - blk * stride;
                const int i = blk * 2 * stride + off;
                cmpswap(i, i + stride);
            }
            tm.sync();
        }
    }
    for (int a = tid; a < newL; a += T) {
        FG_AT(sel, a, NSE) = FG_AT(klist, a, NKL);
        FG_AT(selped, a, NSP) = FG_AT(kped, a, NKP);
    }
#undef NKP
#undef NKL
#undef NSE
#undef NSP
#undef NSW
}

// BK: edge-label planes known at compile time: 0 (unlabelled), 2 (exactly two planes), or
// 8 (any count up to 8, read from the layout)
// CL: the team is a whole cluster (S then lives in global scratch); regions the team
// writes are global, the read-only target-graph tables are per CTA in shared memory.
template <int W, typename MapT, typename Word, int BK, bool CL, typename TS>
__device__ __forceinline__ void solve_pair(const KParams &p, const Regions<Word> R, TS &S,
                                           const int pair)
{
    constexpr int WB = 8 * (int)sizeof(Word);
    const Team<CL> tm;
    const int tid = tm.tid, lane = threadIdx.x & 31, warp = tm.warp;
    const int T = tm.T, NW = tm.NW;
    // CTA-local threads (staging of the per-CTA read-only tables)
    const int ltid = threadIdx.x, LT = blockDim.x;
    const int g1 = FG_AT(p.pairs, 2 * pair, 2 * p.n_pairs);
    const int g2 = FG_AT(p.pairs, 2 * pair + 1, 2 * p.n_pairs);
    const GraphMeta m1 = FG_AT(p.gmeta, g1, p.n_graphs), m2 = FG_AT(p.gmeta, g2, p.n_graphs);
    const int n1 = m1.n, n2 = m2.n, W1 = m1.W, W2 = m2.W;
    const int K = p.kpp ? FG_AT(p.kpp, pair, p.n_pairs) : p.K;
    const int B = BK == 0 ? 0 : (BK == 2 ? 2 : p.lay.B);
    const int N2S = p.lay.n2s;
    const int KM = p.lay.kloc;   // node slots of the P / PL / sbase tables this CTA indexes
    const int64_t mrow = p.lay.mrow;
    const int stride = n2 + 1;   // successors of one node at most: n2 substitutions + deletion
    const MapT DEL = (MapT)~(MapT)0;
    const CostModel c = p.cost;
    const int hwin = p.hwin;     // buckets 0..hwin-2 hold one PED each, hwin-1 the rest
    const bool fold_ie = (c.eins == c.edel);
    // Every successor is one entry of R.cand. Packed classes use 32 bits:
    //   PED << 16 | parent slot << jbits | j,   jbits = bit length of n2 (j = 0..n2);
    // the host packs a class only if no pair's PED can reach 2^16 and every K fits the slot
    // field (K <= 2^(16 - jbits)); single-word classes are always packed. The others use
    // 64 bits: PED << 32 | parent slot << kSelShift | j (the low half is the selection code).
    const bool pk = CL ? false : (W == 1 ? true : p.lay.pk != 0);
    const int jbits = 32 - __clz(n2);
    const uint32_t jmask = (1u << jbits) - 1u;
    uint32_t *ck = (uint32_t *)R.cand;
    uint64_t *ck64 = (uint64_t *)R.cand;
    // lane-constant masks: lane b answers for histogram bucket b
    unsigned lanebit[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) lanebit[k] = ((lane >> k) & 1) ? 0xffffffffu : 0u;
#ifdef FASTGED_PHASE_TIMERS
    long long ph[16] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    long long ph_last = clock64();
#endif

    // stage g2: transposed adjacency and label planes, vertex labels; g1 degrees (these
    // tables are per CTA)
    {
        const uint64_t *adj2 = p.adj + m2.adj_off;
        for (int idx = ltid; idx < W * n2; idx += LT) {
            const int w = idx / n2, u = idx - w * n2;
            const int w64 = (w * WB) >> 6, sh = (w * WB) & 63;
            FG_AT(R.a2t, w * N2S + u, FG_N(Word, p.lay.rsize[RG_A2T])) =
                (w64 < W2) ? (Word)(FG_AT(adj2, (int64_t)u * W2 + w64, p.adj_words - m2.adj_off) >> sh)
                           : (Word)0;
        }
        for (int b = 0; b < B; ++b) {
            const uint64_t *pl2 = p.planes + m2.plane_off + (int64_t)b * n2 * W2;
            for (int idx = ltid; idx < W * n2; idx += LT) {
                const int w = idx / n2, u = idx - w * n2;
                const int w64 = (w * WB) >> 6, sh = (w * WB) & 63;
                FG_AT(R.l2t, (b * W + w) * N2S + u, FG_N(Word, p.lay.rsize[RG_L2T])) =
                    (w64 < W2) ? (Word)(FG_AT(pl2, (int64_t)u * W2 + w64,
                                              p.plane_words - m2.plane_off - (int64_t)b * n2 * W2) >> sh)
                               : (Word)0;
            }
        }
        for (int u = ltid; u < n2; u += LT)
            FG_AT(R.alpha2, u, FG_N(int32_t, p.lay.rsize[RG_ALPHA2])) = FG_AT(p.vlab, m2.lab_off + u, p.n_vlab);
        // column n2 of the target tables is the deletion v_i -> eps: no g2 neighbours, so the
        // substitution formula scores it with the deletion's edge costs (see succ_ped)
        for (int w = ltid; w < W; w += LT) FG_AT(R.a2t, w * N2S + n2, FG_N(Word, p.lay.rsize[RG_A2T])) = (Word)0;
        for (int x = ltid; x < B * W; x += LT) FG_AT(R.l2t, x * N2S + n2, FG_N(Word, p.lay.rsize[RG_L2T])) = (Word)0;
        // S1 cost row of level 0 (the row of level i + 1 is written during level i)
        if (n1 > 0) {
            const int a10 = FG_AT(p.vlab, m1.lab_off, p.n_vlab);
            for (int u = ltid; u <= n2; u += LT)
                FG_AT(R.crow, u, FG_N(int32_t, p.lay.rsize[RG_CROW])) =
                    u < n2 ? ((FG_AT(p.vlab, m2.lab_off + u, p.n_vlab) != a10) ? c.vsub : 0) : c.vdel;
        }
        // number of neighbours v_k of v_i with k < i
        for (int v = ltid; v < n1; v += LT) {
            const int64_t row = m1.adj_off + (int64_t)v * W1;
            int d = 0;
            for (int w = 0; w < W1; ++w)
                d += __popcll(FG_AT(p.adj, row + w, p.adj_words) & low_mask(v, w));
            FG_AT(R.noff, v + 1, FG_N(int32_t, p.lay.rsize[RG_NOFF])) = d;
        }
        if (ltid == 0) FG_AT(R.noff, 0, FG_N(int32_t, p.lay.rsize[RG_NOFF])) = 0;
        // root node: empty lambda, R_V2 = V2, PED 0
        for (int w = tid; w < W; w += T) FG_AT(R.img0, w, FG_N(Word, p.lay.rsize[RG_IMG0])) = (Word)0;
        if (tid == 0) FG_AT(R.ped0, 0, FG_N(int32_t, p.lay.rsize[RG_PED0])) = 0;
    }
    __syncthreads();
    // prior-neighbour lists of g1: nbr[noff[i] .. noff[i+1]) = k | (edge label << 16)
    if (ltid < 32) {
        int carry = 0;
        for (int v0 = 0; v0 < n1; v0 += 32) {
            const int v = v0 + lane;
            const int d = v < n1 ? FG_AT(R.noff, v + 1, FG_N(int32_t, p.lay.rsize[RG_NOFF])) : 0;
            int incl = d;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (v < n1) FG_AT(R.noff, v + 1, FG_N(int32_t, p.lay.rsize[RG_NOFF])) = carry + incl;
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
    __syncthreads();
    for (int v = ltid; v < n1; v += LT) {
        const int64_t row = m1.adj_off + (int64_t)v * W1;
        const int64_t pl = m1.plane_off + (int64_t)v * W1;
        const int64_t pstep = (int64_t)n1 * W1;
        int o = FG_AT(R.noff, v, FG_N(int32_t, p.lay.rsize[RG_NOFF]));
        for (int w = 0; w < W1; ++w) {
            uint64_t bits = FG_AT(p.adj, row + w, p.adj_words) & low_mask(v, w);
            while (bits) {
                const int t = __ffsll((long long)bits) - 1;
                bits &= bits - 1ull;
                int lab = 0;
                for (int b = 0; b < B; ++b)
                    lab |= (int)((FG_AT(p.planes, pl + b * pstep + w, p.plane_words) >> t) & 1ull) << b;
                FG_AT(R.nbr, o++, FG_N(int32_t, p.lay.rsize[RG_NBR])) = (w * 64 + t) | (lab << 16);
            }
        }
    }
    long long nevals = 0;
    int L = 1;
    // current / next beam buffers, swapped after every level
    uint8_t *mapc = R.map0, *mapn = R.map1;
    Word *imgc = R.img0, *imgn = R.img1;
    int32_t *pedc = R.ped0, *pedn = R.ped1;
    int32_t *crc = R.crow, *crn = R.crow + N2S;   // S1 cost rows of this level and the next
    // elements of the beam buffers (both buffers of a pair have the same size), the cost-row
    // halves, the P / PL / sbase tables, the maps in MapT and 16-byte units, the entries
#define NIMG FG_N(Word, p.lay.rsize[RG_IMG0])
#define NPED FG_N(int32_t, p.lay.rsize[RG_PED0])
#define NSW ((int64_t)(sizeof(S.wn) / sizeof(S.wn[0])))   // warps the team scalars hold
#define NP FG_N(Word, p.lay.rsize[RG_P])
#define NMAPT FG_N(MapT, p.lay.rsize[RG_MAP0])
#define NMAP16 FG_N(uint4, p.lay.rsize[RG_MAP0])
#define NCK FG_N(uint32_t, p.lay.rsize[RG_CAND])
#define NCK64 FG_N(uint64_t, p.lay.rsize[RG_CAND])
#define NIMGW (CL ? FG_N(Word, p.lay.rsize[RG_IMGL]) : NIMG)
    tm.sync();
    PHASE_MARK(0);

    for (int i = 0; i < n1; ++i) {
        const int n0 = FG_AT(R.noff, i, FG_N(int32_t, p.lay.rsize[RG_NOFF])), deg = FG_AT(R.noff, i + 1, FG_N(int32_t, p.lay.rsize[RG_NOFF])) - n0;
        const int s_lo = (warp * L) / NW, s_hi = ((warp + 1) * L) / NW;
        const int base = s_lo * stride;              // this warp's successor storage
        // node tables the warp prepares and evaluates are indexed from cs0: 0 for a one-CTA
        // team; for a cluster, the first node of this CTA (its P, PL and sbase are CTA-local
        // and its nodes' Img rows are staged into shared memory)
        int cs0 = 0, ioff = 0;
        const Word *imgw = imgc;
        if (CL) {
            const int nwl = (int)blockDim.x >> 5;
            const int r0 = (int)cluster_rank() * nwl;
            cs0 = (r0 * L) / NW;
            const int cs1 = ((r0 + nwl) * L) / NW;
            for (int x = ltid; x < (cs1 - cs0) * W; x += LT)
                FG_AT(R.imgl, x, FG_N(Word, p.lay.rsize[RG_IMGL])) = FG_AT(imgc, (int64_t)cs0 * W + x, NIMG);
            __syncthreads();
            imgw = R.imgl;
            ioff = cs0;
        }
        // ---- S1 + S2 per-node vectors, successor lists, S3 evaluation ----------------
        int kw = 0;          // successors of this warp so far
        int wmin = INT_MAX;  // least PED this warp scored
        // PED of successor idx
        auto ped_at = [&](int idx) -> int { return entry_ped(p, R.cand, idx, pk); };
        // S3: PED of successor (node sc, column j). Column j == n2 is the deletion
        // v_i -> eps: its A2 column is empty, so the implied-edge terms count every
        // substituted neighbour in P as a deleted edge (with the dcnt deleted neighbours in
        // sbase, all deg edges to v_0..v_{i-1}), and the cost row holds c_vdel there.
        // successors scored during the id sweep (one-CTA teams, two to four words), else in
        // a chunked pass
        constexpr bool kFuseEval = !CL && W > 1 && W <= 4;
        auto succ_ped = [&](int sc, int j) -> int {
            const int64_t im = (int64_t)(sc - ioff) * W;   // the parent's Img row
            const int64_t Ps = (int64_t)(sc - cs0) * W;    // and its row of R.P
            int x = 0, y = 0, z = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const Word aw = FG_AT(R.a2t, w * N2S + j, FG_N(Word, p.lay.rsize[RG_A2T]));
                const Word ai = aw & FG_AT(imgw, im + w, NIMGW);
                const Word pw = FG_AT(R.P, Ps + w, NP);
                if (fold_ie) {
                    x += popcw((Word)(ai ^ pw));
                } else {
                    x += popcw((Word)(ai & ~pw));
                    y += popcw((Word)(pw & ~aw));
                }
                if (B > 0) {
                    Word ld = (Word)0;
                    for (int b = 0; b < B; ++b)
                        ld |= FG_AT(R.PL, ((int64_t)b * KM + (sc - cs0)) * W + w, FG_N(Word, p.lay.rsize[RG_PL])) ^
                              FG_AT(R.l2t, (b * W + w) * N2S + j, FG_N(Word, p.lay.rsize[RG_L2T]));
                    z += popcw((Word)(aw & pw & ld));
                }
            }
            return FG_AT(R.sbase, sc - cs0, FG_N(int32_t, p.lay.rsize[RG_SBASE])) + FG_AT(crc, j, N2S) +
                   c.eins * x + c.edel * y + c.esub * z;
        };
        for (int g0 = s_lo; g0 < s_hi; g0 += 32) {
            const int ng = min(32, s_hi - g0);
            const int s = g0 + lane;
            const bool act = lane < ng;
            int cnt = 0;
            if (act) {
                // S2: P = images of the substituted g1 neighbours of v_i (their edge labels in
                // bit-planes PL at the image positions); dcnt = deleted neighbours
                const int64_t Ps = (int64_t)(s - cs0) * W;   // this node's row of R.P
                const int64_t ms = (int64_t)s * (mrow / (int64_t)sizeof(MapT));   // its map row
                int dcnt = 0;
                if (W == 1) {
                    constexpr int NPL = BK == 8 ? kMaxB : (BK == 2 ? 2 : 1);
                    Word pr = (Word)0, plr[NPL];
#pragma unroll
                    for (int b = 0; b < NPL; ++b) plr[b] = (Word)0;
                    // four neighbours per step: list and map loads first, then the bits
                    for (int t0 = 0; t0 < deg; t0 += 4) {
                        int e[4];
                        MapT phi[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) e[u] = t0 + u < deg ? FG_AT(R.nbr, n0 + t0 + u, FG_N(int32_t, p.lay.rsize[RG_NBR])) : -1;
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            phi[u] = e[u] >= 0 ? FG_AT((const MapT *)mapc, ms + (e[u] & 0xffff), NMAPT) : DEL;
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const bool sub = phi[u] != DEL;
                            dcnt += (e[u] >= 0 && !sub) ? 1 : 0;
                            const Word pb = sub ? (Word)1 << ((int)phi[u] % WB) : (Word)0;
                            pr |= pb;
#pragma unroll
                            for (int b = 0; b < NPL; ++b)
                                if (b < B && ((e[u] >> (16 + b)) & 1)) plr[b] |= pb;
                        }
                    }
                    FG_AT(R.P, Ps, NP) = pr;
#pragma unroll
                    for (int b = 0; b < NPL; ++b)
                        if (b < B) FG_AT(R.PL, (int64_t)b * KM + (s - cs0), FG_N(Word, p.lay.rsize[RG_PL])) = plr[b];
                } else {
#pragma unroll
                    for (int w = 0; w < W; ++w) FG_AT(R.P, Ps + w, NP) = (Word)0;
                    for (int b = 0; b < B; ++b)
                        for (int w = 0; w < W; ++w) FG_AT(R.PL, ((int64_t)b * KM + (s - cs0)) * W + w, FG_N(Word, p.lay.rsize[RG_PL])) = (Word)0;
                    for (int t = 0; t < deg; ++t) {
                        const int e = FG_AT(R.nbr, n0 + t, FG_N(int32_t, p.lay.rsize[RG_NBR]));
                        const MapT phi = FG_AT((const MapT *)mapc, ms + (e & 0xffff), NMAPT);
                        if (phi == DEL) { ++dcnt; continue; }
                        const int pw = (int)phi / WB;
                        const Word pb = (Word)1 << ((int)phi % WB);
                        FG_AT(R.P, Ps + pw, NP) |= pb;
                        for (int b = 0; b < B; ++b)
                            if ((e >> (16 + b)) & 1) FG_AT(R.PL, ((int64_t)b * KM + (s - cs0)) * W + pw, FG_N(Word, p.lay.rsize[RG_PL])) |= pb;
                    }
                }
                FG_AT(R.sbase, s - cs0, FG_N(int32_t, p.lay.rsize[RG_SBASE])) =
                    FG_AT(pedc, s, NPED) + c.edel * dcnt;
                const int64_t im = (int64_t)(s - ioff) * W;   // this node's Img row in imgw
                int used = 0;
#pragma unroll
                for (int w = 0; w < W; ++w) used += popcw(FG_AT(imgw, im + w, NIMGW));
                cnt = n2 - used + 1;   // free g2 vertices (R_V2) and the deletion
            }
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const int excl = incl - cnt;
            const int gtot = __shfl_sync(0xffffffffu, incl, 31);
            // successor ids in enumeration order: for each node the free g2 vertices in
            // increasing order, then n2 for v_i -> eps. Single-word bitsets: each lane walks
            // its own node's bits; wider ones: the warp sweeps each node's vertices 32 at a
            // time and compacts the free ones with a ballot.
            if (W == 1 && !CL) {
                if (act) {
                    int idx = base + kw + excl;
                    Word x = ~FG_AT(imgw, (int64_t)(s - ioff) * W, NIMGW);
                    if (n2 < WB) x &= n2 > 0 ? (((Word)1 << n2) - (Word)1) : (Word)0;
                    while (x) {
                        const int t = (WB == 64) ? __ffsll((long long)x) - 1 : __ffs((int)x) - 1;
                        x &= x - (Word)1;
                        FG_AT(ck, idx, NCK) = ((uint32_t)s << jbits) | (uint32_t)t;
                        ++idx;
                    }
                    FG_AT(ck, idx, NCK) = ((uint32_t)s << jbits) | (uint32_t)n2;
                }
            } else {
                // one-CTA teams with two to four words: the sweep scores each free vertex
                // where it finds it and writes the whole entry (PED and id), so the entries
                // are not read back for the evaluation. Otherwise it writes ids, scored by the
                // chunked pass below, where every lane scores a free vertex: that pays off
                // once an evaluation costs eight words, and for cluster teams, whose pairs
                // (wide beams) can have fewer target vertices than a warp has lanes
                __syncwarp();   // the group's node vectors (P, PL, base) are in place
                for (int t = 0; t < ng; ++t) {
                    const int st_ = g0 + t;
                    const int64_t im = (int64_t)(st_ - ioff) * W;   // the node's Img row
                    const int o0 = base + kw + __shfl_sync(0xffffffffu, excl, t);
                    int pos = 0;
                    for (int j0 = 0; j0 < n2; j0 += 32) {
                        const int j = j0 + lane;
                        const bool fr = j < n2 && !((FG_AT(imgw, im + j / WB, NIMGW) >> (j % WB)) & (Word)1);
                        const unsigned bal = __ballot_sync(0xffffffffu, fr);
                        if (fr) {
                            const int idx = o0 + pos + __popc(bal & lanemask_lt());
                            const int d = kFuseEval ? succ_ped(st_, j) : 0;
                            if (kFuseEval) wmin = d < wmin ? d : wmin;
                            if (pk) FG_AT(ck, idx, NCK) = ((uint32_t)d << 16) | ((uint32_t)st_ << jbits) | (uint32_t)j;
                            else FG_AT(ck64, idx, NCK64) = ((uint64_t)(uint32_t)d << 32) | ((uint64_t)st_ << kSelShift) | (uint64_t)j;
                        }
                        pos += __popc(bal);
                    }
                    if (lane == 0) {
                        const int d = kFuseEval ? succ_ped(st_, n2) : 0;
                        if (kFuseEval) wmin = d < wmin ? d : wmin;
                        if (pk) FG_AT(ck, o0 + pos, NCK) = ((uint32_t)d << 16) | ((uint32_t)st_ << jbits) | (uint32_t)n2;
                        else FG_AT(ck64, o0 + pos, NCK64) = ((uint64_t)(uint32_t)d << 32) | ((uint64_t)st_ << kSelShift) | (uint64_t)n2;
                    }
                }
            }
            __syncwarp();
            PHASE_MARK(5);

            // U chunks of 32 successors per step, their id loads and PEDs independent
            constexpr int U = 2;
            for (int kb = 0; !kFuseEval && kb < gtot; kb += 32 * U) {
                int scu[U], ju[U];
                uint32_t idu[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int k = kb + 32 * u + lane;
                    const int idx = base + kw + k;
                    if (pk) {
                        idu[u] = k < gtot ? FG_AT(ck, idx, NCK) : (((uint32_t)g0 << jbits) | (uint32_t)n2);
                        scu[u] = (int)(idu[u] >> jbits);
                        ju[u] = (int)(idu[u] & jmask);
                    } else {
                        idu[u] = k < gtot ? (uint32_t)FG_AT(ck64, idx, NCK64)
                                          : (((uint32_t)g0 << kSelShift) | (uint32_t)n2);
                        scu[u] = (int)(idu[u] >> kSelShift);
                        ju[u] = (int)(idu[u] & ((1u << kSelShift) - 1u));
                    }
                }
                int pu[U];
#pragma unroll
                for (int u = 0; u < U; ++u) pu[u] = succ_ped(scu[u], ju[u]);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int k = kb + 32 * u + lane;
                    if (k < gtot) {
                        if (pk) FG_AT(ck, base + kw + k, NCK) = ((uint32_t)pu[u] << 16) | idu[u];
                        else FG_AT(ck64, base + kw + k, NCK64) = ((uint64_t)(uint32_t)pu[u] << 32) | idu[u];
                        wmin = pu[u] < wmin ? pu[u] : wmin;
                    }
                }
            }
            kw += gtot;
            __syncwarp();
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wmin = min(wmin, __shfl_xor_sync(0xffffffffu, wmin, o));
        if (lane == 0) {
            FG_AT(S.wmin, warp, NSW) = wmin;
            FG_AT(S.wn, warp, NSW) = kw;
        }
        tm.sync();
        // S4 histogram of PED - pa over this warp's successors, pa = least PED of the level
        // (the last bucket collects every PED past the window). Ballot counting: lane b keeps
        // the count of bucket b; lanes past the end count in the last bucket, which only
        // bounds the threshold search from above (the level total comes from the counts kw).
        int pa = INT_MAX;
        for (int w = lane; w < NW; w += 32) pa = min(pa, FG_AT(S.wmin, w, NSW));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pa = min(pa, __shfl_xor_sync(0xffffffffu, pa, o));
        {
            int hreg = 0;
            if (kw >= 1024 && kw <= 65000) {
                // many candidates: each lane counts its own in 4-bit fields (two 64-bit words
                // for 32 buckets), widened every 12 chunks into 16-bit fields, then a five-
                // round shuffle reduce-scatter leaves bucket b's warp total in lane b (16-bit
                // fields hold it: the warp has at most 65,000 candidates plus padding)
                unsigned long long c0 = 0ull, c1 = 0ull, acc[8];
#pragma unroll
                for (int m = 0; m < 8; ++m) acc[m] = 0ull;
                int pending = 0;
                for (int kb = 0; kb < kw; kb += 128) {
                    int d4[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int k = kb + 32 * u + lane;
                        d4[u] = k < kw ? min(ped_at(base + k) - pa, hwin - 1) : hwin - 1;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const unsigned long long inc = 1ull << (4 * (d4[u] & 15));
                        if (d4[u] < 16) c0 += inc; else c1 += inc;
                    }
                    pending += 4;
                    if (pending >= 12 || kb + 128 >= kw) {
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            acc[m] += (c0 >> (4 * m)) & 0x000F000F000F000Full;
                            acc[4 + m] += (c1 >> (4 * m)) & 0x000F000F000F000Full;
                        }
                        c0 = c1 = 0ull;
                        pending = 0;
                    }
                }
                const bool b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1, b2 = (lane >> 2) & 1;
                const bool b1 = (lane >> 1) & 1, b0 = lane & 1;
                unsigned q[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const unsigned long long send = b4 ? acc[m] : acc[4 + m];
                    const unsigned long long keep = b4 ? acc[4 + m] : acc[m];
                    const unsigned long long r = keep + __shfl_xor_sync(0xffffffffu, send, 16);
                    const unsigned lo = (unsigned)r, hi = (unsigned)(r >> 32);
                    q[m] = (b3 ? hi : lo) + __shfl_xor_sync(0xffffffffu, b3 ? lo : hi, 8);
                }
                unsigned t[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const unsigned lo = q[m] & 0xffffu, hi = q[m] >> 16;
                    t[m] = (b2 ? hi : lo) + __shfl_xor_sync(0xffffffffu, b2 ? lo : hi, 4);
                }
                unsigned u2[2];
#pragma unroll
                for (int m = 0; m < 2; ++m)
                    u2[m] = (b1 ? t[2 + m] : t[m]) + __shfl_xor_sync(0xffffffffu, b1 ? t[m] : t[2 + m], 2);
                hreg = (int)((b0 ? u2[1] : u2[0]) + __shfl_xor_sync(0xffffffffu, b0 ? u2[0] : u2[1], 1));
            } else
            // few candidates: five bit ballots per chunk, lane b counts the lanes whose
            // bucket is b
            for (int kb = 0; kb < kw; kb += 128) {
                int d4[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = kb + 32 * u + lane;
                    d4[u] = k < kw ? min(ped_at(base + k) - pa, hwin - 1) : hwin - 1;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (kb + 32 * u >= kw) break;
                    unsigned m = 0xffffffffu;
#pragma unroll
                    for (int b = 0; b < 5; ++b)
                        m &= ~(__ballot_sync(0xffffffffu, (d4[u] >> b) & 1) ^ lanebit[b]);
                    hreg += __popc(m);
                }
            }
            FG_AT(R.hist, lane * NW + warp, FG_N(int32_t, p.lay.rsize[RG_HIST])) = hreg;
        }
        tm.sync();
        PHASE_MARK(1);
        // (parent slot << kSelShift) | j of successor idx
        auto decode = [&](int idx) -> int {
            if (pk) {
                const uint32_t id = FG_AT(ck, idx, NCK) & 0xffffu;
                return (int)((id >> jbits) << kSelShift) | (int)(id & jmask);
            } else {
                return (int)(uint32_t)FG_AT(ck64, idx, NCK64);
            }
        };

        if (p.variant == 1 && i == n1 - 1) {
            // variant B: every successor of the last level is completed (insertions of the
            // free g2 vertices and their edges) and the least (total, PED, enumeration order)
            // wins. Per node: nimg = |Img|, e2 = g2 edges inside Img (kept in klist / kped,
            // which the selection does not use at this level).
            for (int t = lane; t < s_hi - s_lo; t += 32) {
                const int sl = s_lo + t;
                const int64_t im = (int64_t)sl * W;   // the node's Img row
                int nimg = 0, acc = 0;
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    Word x = FG_AT(imgc, im + w, NIMG);
                    nimg += popcw(x);
                    while (x) {
                        const int bt = (WB == 64) ? __ffsll((long long)x) - 1 : __ffs((int)x) - 1;
                        x &= x - (Word)1;
                        const int u = w * WB + bt;
#pragma unroll
                        for (int w2 = 0; w2 < W; ++w2)
                            acc += popcw((Word)(FG_AT(R.a2t, w2 * N2S + u, FG_N(Word, p.lay.rsize[RG_A2T])) &
                                                FG_AT(imgc, im + w2, NIMG)));
                    }
                }
                FG_AT(R.kped, sl, FG_N(int32_t, p.lay.rsize[RG_KPED])) = nimg;
                FG_AT(R.klist, sl, FG_N(int32_t, p.lay.rsize[RG_KLIST])) = acc / 2;
            }
            __syncwarp();
            auto leaf_total = [&](int k) -> long long {
                const int idx = base + k;
                const int v = decode(idx);
                const int sc = v >> kSelShift, j = v & ((1 << kSelShift) - 1);
                const int64_t im = (int64_t)sc * W;   // the parent's Img row
                int nimg = FG_AT(R.kped, sc, FG_N(int32_t, p.lay.rsize[RG_KPED])), e2 = FG_AT(R.klist, sc, FG_N(int32_t, p.lay.rsize[RG_KLIST]));
                if (j < n2) {
                    ++nimg;
#pragma unroll
                    for (int w = 0; w < W; ++w)
                        e2 += popcw((Word)(FG_AT(R.a2t, w * N2S + j, FG_N(Word, p.lay.rsize[RG_A2T])) &
                                           FG_AT(imgc, im + w, NIMG)));
                }
                return (long long)ped_at(idx) + (long long)c.vins * (n2 - nimg) +
                       (long long)c.eins * (m2.m - e2);
            };
            long long tmin = LLONG_MAX;
            for (int k = lane; k < kw; k += 32) tmin = min(tmin, leaf_total(k));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) tmin = min(tmin, (long long)__shfl_xor_sync(0xffffffffu, tmin, o));
            if (lane == 0) FG_AT(S.wbest, warp, NSW) = (unsigned long long)tmin;
            tm.sync();
            long long best_total = LLONG_MAX;
            for (int w = 0; w < NW; ++w) best_total = min(best_total, (long long)FG_AT(S.wbest, w, NSW));
            tm.sync();
            unsigned long long key = ~0ull;
            for (int k = lane; k < kw; k += 32)
                if (leaf_total(k) == best_total) {
                    const unsigned long long kk =
                        ((unsigned long long)ped_at(base + k) << 32) | (unsigned)(base + k);
                    key = kk < key ? kk : key;
                }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long y = __shfl_xor_sync(0xffffffffu, key, o);
                key = y < key ? y : key;
            }
            if (lane == 0) FG_AT(S.wbest, warp, NSW) = key;
            tm.sync();
            unsigned long long bk = FG_AT(S.wbest, 0, NSW);
            for (int w = 1; w < NW; ++w) bk = FG_AT(S.wbest, w, NSW) < bk ? FG_AT(S.wbest, w, NSW) : bk;
            const int widx = (int)(bk & 0xffffffffull);
            const int wv = decode(widx);
            const int ws = wv >> kSelShift, wj = wv & ((1 << kSelShift) - 1);
            int all = 0;
            for (int w = 0; w < NW; ++w) all += FG_AT(S.wn, w, NSW);
            if (tid == 0) {
                FG_AT(p.out_cost, pair, p.n_pairs) = (int32_t)best_total;
                if (p.out_nevals) FG_AT(p.out_nevals, pair, p.n_pairs) = nevals + 2LL * all;
            }
            const int64_t mb = (int64_t)ws * (mrow / (int64_t)sizeof(MapT));   // the winner's map row
            const int64_t om = FG_AT(p.map_off, pair, p.n_pairs);
            for (int k = tid; k < n1; k += T) {
                const MapT v = (k == i) ? ((wj < n2) ? (MapT)wj : DEL) : FG_AT((const MapT *)mapc, mb + k, NMAPT);
                FG_AT(p.out_map, om + k, p.map_total) = (v == DEL) ? -1 : (int32_t)v;
            }
            tm.sync();
            return;
        }

        // ---- S4 selection ---------------------------------------------------------
        // every warp reads the (bucket, warp) table: bucket totals, their exclusive prefix,
        // and the bucket-b successors of the warps before this one; eight loads in flight
        // per lane (a cluster team's table is in global scratch)
        int tot = 0, mine = 0;
        {
            const int64_t hb = (int64_t)lane * NW;
            int w = 0;
            for (; w + 8 <= NW; w += 8) {
                int v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = FG_AT(R.hist, hb + w + u, FG_N(int32_t, p.lay.rsize[RG_HIST]));
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    tot += v[u];
                    mine += (w + u < warp) ? v[u] : 0;
                }
            }
            for (; w < NW; ++w) {
                const int v = FG_AT(R.hist, hb + w, FG_N(int32_t, p.lay.rsize[RG_HIST]));
                tot += v;
                mine += (w < warp) ? v : 0;
            }
        }
        int incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int bexcl = incl - tot;
        int total = 0;   // successors of the level (the last bucket may hold padding)
        for (int w = lane; w < NW; w += 32) total += FG_AT(S.wn, w, NSW);
        total = warp_sum(total);
        const int newL = min(K, total);
        // the bucket where the cumulative count reaches newL
        const int thr = __ffs(__ballot_sync(0xffffffffu, bexcl < newL && incl >= newL)) - 1;
        if (tid == 0) nevals += total;
        PHASE_MARK(2);
        if (thr < hwin - 1) {
            // kept = every successor below the threshold bucket and the first q in it. Each
            // warp compacts its kept successors in enumeration order, then places them at
            // their rank in (PED, parent slot, j) order: position = #(smaller PED) +
            // #(equal PED earlier); lane b holds the bucket-b counts of earlier warps.
            const int q = newL - __shfl_sync(0xffffffffu, bexcl, thr);
            const int eq_before = __shfl_sync(0xffffffffu, mine, thr);
            const int lt_before = warp_sum(lane < thr ? mine : 0);
            const int kbeg = lt_before + min(q, eq_before);
            const int kcnt = compact_kept<Word>(p, R, base, kw, pa + thr, q, kbeg, eq_before, pk);
            __syncwarp();
            PHASE_MARK(8);
            int run = lane < thr ? mine : min(q, eq_before);   // kept of bucket `lane` before
            for (int xb = 0; xb < kcnt; xb += 32) {
                const int x = kbeg + xb + lane;
                const bool v = xb + lane < kcnt;
                const int d = v ? FG_AT(R.kped, x, FG_N(int32_t, p.lay.rsize[RG_KPED])) - pa : 0;
                const unsigned V = __ballot_sync(0xffffffffu, v);
                unsigned bb[5];
#pragma unroll
                for (int b = 0; b < 5; ++b) bb[b] = __ballot_sync(0xffffffffu, (d >> b) & 1);
                const int pos = __shfl_sync(0xffffffffu, bexcl, d) +
                                __shfl_sync(0xffffffffu, run, d) +
                                __popc(same_value_lanes(V, bb, d) & lanemask_lt());
                if (v) {
                    FG_AT(R.sel, pos, FG_N(int32_t, p.lay.rsize[RG_SEL])) = decode(FG_AT(R.klist, x, FG_N(int32_t, p.lay.rsize[RG_KLIST])));
                    FG_AT(R.selped, pos, FG_N(int32_t, p.lay.rsize[RG_SELPED])) = d + pa;
                }
                unsigned m = V;
#pragma unroll
                for (int b = 0; b < 5; ++b) m &= ~(bb[b] ^ lanebit[b]);
                run += __popc(m);
            }
            PHASE_MARK(9);
        } else {
#ifdef FASTGED_PHASE_TIMERS
            if (threadIdx.x == 0) ph[7] += 1;   // levels that took the exact selection
#endif
            select_exact<MapT, Word, CL, TS>(p, R.cand, R.klist, R.kped, R.sel, R.selped, S, L,
                                             stride, newL, pa + hwin - 1, pk);
            tm.sync();
            for (int r = tid; r < newL; r += T) FG_AT(R.sel, r, FG_N(int32_t, p.lay.rsize[RG_SEL])) = decode(FG_AT(R.sel, r, FG_N(int32_t, p.lay.rsize[RG_SEL])));
        }
        tm.sync();
        PHASE_MARK(6);

        // ---- kept children, in key order (slot = rank) -----------------------------
        {
            const int nvec = (int)((i * (int)sizeof(MapT) + 15) >> 4);
            const int64_t m16 = mrow >> 4, mt = mrow / (int64_t)sizeof(MapT);   // a map row in
                                                                                // 16 B / MapT units
            if (mrow <= 128) {
                for (int r = tid; r < newL; r += T) {
                    const int v = FG_AT(R.sel, r, FG_N(int32_t, p.lay.rsize[RG_SEL]));
                    const int s = v >> kSelShift, j = v & ((1 << kSelShift) - 1);
                    for (int t = 0; t < nvec; ++t)
                        FG_AT((uint4 *)mapn, r * m16 + t, NMAP16) = FG_AT((const uint4 *)mapc, s * m16 + t, NMAP16);
                    FG_AT((MapT *)mapn, r * mt + i, NMAPT) = (j < n2) ? (MapT)j : DEL;
#pragma unroll
                    for (int w = 0; w < W; ++w) {
                        Word x = FG_AT(imgc, (int64_t)s * W + w, NIMG);
                        if (j < n2 && j / WB == w) x |= (Word)1 << (j % WB);
                        FG_AT(imgn, (int64_t)r * W + w, NIMG) = x;
                    }
                    FG_AT(pedn, r, NPED) = FG_AT(R.selped, r, FG_N(int32_t, p.lay.rsize[RG_SELPED]));
                }
            } else if (!CL) {
                // long maps, one-CTA team: every thread takes (child, 16-byte vector) items
                // (the last vector of a child also carries its new entry i) and one more item
                // per child writes Img, the PED and entry i when it starts a new vector
                const int nb = i * (int)sizeof(MapT);
                const int per = nvec + 1;
                const int items = newL * per;
                for (int t = tid; t < items; t += T) {
                    const int r = t / per, v = t - r * per;
                    const int sv = FG_AT(R.sel, r, FG_N(int32_t, p.lay.rsize[RG_SEL]));
                    const int s = sv >> kSelShift, j = sv & ((1 << kSelShift) - 1);
                    const MapT val = (j < n2) ? (MapT)j : DEL;
                    if (v < nvec) {
                        uint4 x = FG_AT((const uint4 *)mapc, s * m16 + v, NMAP16);
                        if (v == nvec - 1 && nb < 16 * nvec)
                            ((MapT *)&x)[(nb - 16 * v) / (int)sizeof(MapT)] = val;
                        FG_AT((uint4 *)mapn, r * m16 + v, NMAP16) = x;
                    } else {
                        if (nb == 16 * nvec) FG_AT((MapT *)mapn, r * mt + i, NMAPT) = val;
                        for (int w = 0; w < W; ++w) {
                            Word x = FG_AT(imgc, (int64_t)s * W + w, NIMG);
                            if (j < n2 && j / WB == w) x |= (Word)1 << (j % WB);
                            FG_AT(imgn, (int64_t)r * W + w, NIMG) = x;
                        }
                        FG_AT(pedn, r, NPED) = FG_AT(R.selped, r, FG_N(int32_t, p.lay.rsize[RG_SELPED]));
                    }
                }
            } else {
                // cluster teams: a warp per child
                for (int r = warp; r < newL; r += NW) {
                    const int v = FG_AT(R.sel, r, FG_N(int32_t, p.lay.rsize[RG_SEL]));
                    const int s = v >> kSelShift, j = v & ((1 << kSelShift) - 1);
                    for (int t = lane; t < nvec; t += 32)
                        FG_AT((uint4 *)mapn, r * m16 + t, NMAP16) = FG_AT((const uint4 *)mapc, s * m16 + t, NMAP16);
                    for (int w = lane; w < W; w += 32) {
                        Word x = FG_AT(imgc, (int64_t)s * W + w, NIMG);
                        if (j < n2 && j / WB == w) x |= (Word)1 << (j % WB);
                        FG_AT(imgn, (int64_t)r * W + w, NIMG) = x;
                    }
                    __syncwarp();
                    if (lane == 0) {
                        FG_AT((MapT *)mapn, r * mt + i, NMAPT) = (j < n2) ? (MapT)j : DEL;
                        FG_AT(pedn, r, NPED) = FG_AT(R.selped, r, FG_N(int32_t, p.lay.rsize[RG_SELPED]));
                    }
                }
            }
        }
        // S1 cost row of the next level (each CTA keeps its own copy)
        if (i + 1 < n1) {
            const int a1n = FG_AT(p.vlab, m1.lab_off + i + 1, p.n_vlab);
            for (int u = ltid; u <= n2; u += LT)
                FG_AT(crn, u, N2S) = u < n2 ? ((FG_AT(R.alpha2, u, FG_N(int32_t, p.lay.rsize[RG_ALPHA2])) != a1n) ? c.vsub : 0) : c.vdel;
        }
        tm.sync();
        PHASE_MARK(3);
        { int32_t *t = crc; crc = crn; crn = t; }
        { uint8_t *t = mapc; mapc = mapn; mapn = t; }
        { Word *t = imgc; imgc = imgn; imgn = t; }
        { int32_t *t = pedc; pedc = pedn; pedn = t; }
        L = newL;
    }

    // ---- S5 leaf completion (insert the free g2 vertices and their edges) + argmin ------
    {
        unsigned long long best = ~0ull;
        for (int s = warp; s < L; s += NW) {
            const int64_t im = (int64_t)s * W;   // the leaf's Img row
            int acc = 0;
            for (int u = lane; u < n2; u += 32) {
                if ((FG_AT(imgc, im + u / WB, NIMG) >> (u % WB)) & (Word)1) {
#pragma unroll
                    for (int w = 0; w < W; ++w)
                        acc += popcw((Word)(FG_AT(R.a2t, w * N2S + u, FG_N(Word, p.lay.rsize[RG_A2T])) &
                                            FG_AT(imgc, im + w, NIMG)));
                }
            }
            int nimg = 0;
            for (int w = lane; w < W; w += 32) nimg += popcw(FG_AT(imgc, im + w, NIMG));
            acc = warp_sum(acc);
            nimg = warp_sum(nimg);
            // g2 edges with both ends used were counted twice in acc
            const long long total = (long long)FG_AT(pedc, s, NPED) + (long long)c.vins * (n2 - nimg) +
                                    (long long)c.eins * (m2.m - acc / 2);
            const unsigned long long key = ((unsigned long long)total << 32) | (unsigned)s;
            best = key < best ? key : best;
        }
        if (lane == 0) FG_AT(S.wbest, warp, NSW) = best;
        tm.sync();
        if (tid == 0) {
            unsigned long long b = FG_AT(S.wbest, 0, NSW);
            for (int w = 1; w < NW; ++w) b = FG_AT(S.wbest, w, NSW) < b ? FG_AT(S.wbest, w, NSW) : b;
            FG_AT(S.wbest, 0, NSW) = b;
            FG_AT(p.out_cost, pair, p.n_pairs) = (int32_t)(b >> 32);
            if (p.out_nevals) FG_AT(p.out_nevals, pair, p.n_pairs) = nevals + L;
        }
        tm.sync();
        const int bs = (int)(FG_AT(S.wbest, 0, NSW) & 0xffffffffull);
        const int64_t mb = (int64_t)bs * (mrow / (int64_t)sizeof(MapT));   // the winner's map row
        const int64_t om = FG_AT(p.map_off, pair, p.n_pairs);
        for (int k = tid; k < n1; k += T) {
            const MapT v = FG_AT((const MapT *)mapc, mb + k, NMAPT);
            FG_AT(p.out_map, om + k, p.map_total) = (v == DEL) ? -1 : (int32_t)v;
        }
        tm.sync();
        PHASE_MARK(4);
    }
#ifdef FASTGED_PHASE_TIMERS
    if (tid == 0 && p.phase_cycles)
        for (int k = 0; k < 16; ++k) atomicAdd(&p.phase_cycles[k], (unsigned long long)ph[k]);
#endif
#undef NIMG
#undef NPED
#undef NSW
#undef NP
#undef NMAPT
#undef NMAP16
#undef NCK
#undef NCK64
#undef NIMGW
}

// Region pointers of a team from a region -> base address function.
template <typename Word, typename F>
__device__ __forceinline__ Regions<Word> make_regions(F base)
{
    Regions<Word> R;
    R.hist = (int32_t *)base(RG_HIST);
    R.alpha2 = (int32_t *)base(RG_ALPHA2);
    R.crow = (int32_t *)base(RG_CROW);
    R.a2t = (Word *)base(RG_A2T);
    R.l2t = (Word *)base(RG_L2T);
    R.sbase = (int32_t *)base(RG_SBASE);
    R.ped0 = (int32_t *)base(RG_PED0);
    R.ped1 = (int32_t *)base(RG_PED1);
    R.sel = (int32_t *)base(RG_SEL);
    R.selped = (int32_t *)base(RG_SELPED);
    R.klist = (int32_t *)base(RG_KLIST);
    R.kped = (int32_t *)base(RG_KPED);
    R.noff = (int32_t *)base(RG_NOFF);
    R.nbr = (int32_t *)base(RG_NBR);
    R.img0 = (Word *)base(RG_IMG0);
    R.img1 = (Word *)base(RG_IMG1);
    R.P = (Word *)base(RG_P);
    R.PL = (Word *)base(RG_PL);
    R.cand = (int32_t *)base(RG_CAND);
    R.map0 = base(RG_MAP0);
    R.map1 = base(RG_MAP1);
    R.imgl = (Word *)base(RG_IMGL);
    return R;
}

// SM: every region lives in shared memory (addresses then stay in the shared window)
template <int W, typename MapT, typename Word, bool SM, int BK>
__global__ void __launch_bounds__(512, 2) kbest_kernel(const KParams p)
{
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ TeamShared S;
    uint8_t *gs = p.gscratch + (int64_t)blockIdx.x * p.lay.slice_bytes;
    auto base = [&](int r) -> uint8_t * {
        if (SM) return smem + p.lay.off[r];
        return ((p.lay.smem_mask >> r) & 1u ? smem : gs) + p.lay.off[r];
    };
    const Regions<Word> R = make_regions<Word>(base);
    for (;;) {
        if (threadIdx.x == 0) S.pair = atomicAdd(p.queue_head, 1);
        __syncthreads();
        const int qi = S.pair;
        __syncthreads();
        if (qi >= p.n_order) break;
        solve_pair<W, MapT, Word, BK, false, TeamShared>(p, R, S, FG_AT(p.order, qi, p.n_order));
    }
}

// One pair per thread-block cluster: every CTA of the cluster belongs to the team. Each
// CTA keeps its own copy of the read-only target-graph tables; what the team writes lives in
// the cluster's slice of global scratch, together with the team scalars. Two-word teams are
// held to 64 registers so that two CTAs share an SM (more clusters resident at once); wider
// ones keep 128 (their 16-word evaluation would spill).
template <int W, typename MapT, typename Word, int BK>
__global__ void __launch_bounds__(512, (W <= 2) ? 2 : 1) kbest_cluster_kernel(const KParams p)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const unsigned crank = cluster_rank(), csize = cluster_size();
    uint8_t *gs = p.gscratch + (int64_t)(blockIdx.x / csize) * p.lay.slice_bytes;
    uint8_t *gc = gs + p.lay.cta_off + (int64_t)crank * p.lay.cta_bytes;   // this CTA's block
    auto base = [&](int r) -> uint8_t * {
        if ((p.lay.smem_mask >> r) & 1u) return smem + p.lay.off[r];
        return ((p.lay.cta_mask >> r) & 1u ? gc : gs) + p.lay.off[r];
    };
    const Regions<Word> R = make_regions<Word>(base);
    TeamSharedCl &S = *(TeamSharedCl *)(gs + p.lay.team_off);
    for (;;) {
        if (crank == 0 && threadIdx.x == 0) S.pair = atomicAdd(p.queue_head, 1);
        cluster_barrier();
        const int qi = *(volatile int *)&S.pair;
        cluster_barrier();
        if (qi >= p.n_order) break;
        solve_pair<W, MapT, Word, BK, true, TeamSharedCl>(p, R, S, FG_AT(p.order, qi, p.n_order));
    }
}

// ------------------------------------------------------------------------------------
// launch wrappers (host side)
// ------------------------------------------------------------------------------------
// Opts the kernel into the device's full dynamic shared memory (needed above 48 KB) before
// it is launched or queried for occupancy.
template <int W, typename MapT, typename Word, bool SM, int BK>
static cudaError_t ensure_smem_attr()
{
    static bool done = false;
    if (done) return cudaSuccess;
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kbest_kernel<W, MapT, Word, SM, BK>);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kbest_kernel<W, MapT, Word, SM, BK>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) done = true;
    return e;
}

template <int W, typename MapT, typename Word, bool SM, int BK>
static cudaError_t launch_one(const KParams &p, int grid, int block, size_t smem,
                              cudaStream_t st)
{
    cudaError_t e = ensure_smem_attr<W, MapT, Word, SM, BK>();
    if (e != cudaSuccess) return e;
    kbest_kernel<W, MapT, Word, SM, BK><<<grid, block, smem, st>>>(p);
    return cudaGetLastError();
}

template <int W, typename MapT, typename Word, bool SM, int BK>
static cudaError_t occupancy_one(int block, size_t smem, int *out)
{
    cudaError_t e = ensure_smem_attr<W, MapT, Word, SM, BK>();
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, kbest_kernel<W, MapT, Word, SM, BK>,
                                                         block, smem);
}

// size class -> template instance. 16-bit maps only occur with W >= 4 (n2 >= 255), and the
// all-shared-memory variant is built for bitsets of up to 4 words.
#define FASTGED_DISPATCH(W_, wide, w32, sm, CALL)                                        \
    do {                                                                                 \
        if (sm) {                                                                        \
            if (w32) return CALL(1, uint8_t, uint32_t, true);                            \
            if (W_ == 1 && !wide) return CALL(1, uint8_t, uint64_t, true);               \
            if (W_ == 2 && !wide) return CALL(2, uint8_t, uint64_t, true);               \
            if (W_ == 4 && !wide) return CALL(4, uint8_t, uint64_t, true);               \
        }                                                                                \
        if (w32) return CALL(1, uint8_t, uint32_t, false);                               \
        switch (W_) {                                                                    \
        case 1: if (!wide) return CALL(1, uint8_t, uint64_t, false); break;              \
        case 2: if (!wide) return CALL(2, uint8_t, uint64_t, false); break;              \
        case 4: if (wide) return CALL(4, uint16_t, uint64_t, false);                     \
                else return CALL(4, uint8_t, uint64_t, false);                           \
        case 8: return CALL(8, uint16_t, uint64_t, false);                               \
        case 16: return CALL(16, uint16_t, uint64_t, false);                             \
        default: break;                                                                  \
        }                                                                                \
        return cudaErrorInvalidValue;                                                    \
    } while (0)

template <int W, typename MapT, typename Word, int BK>
static cudaError_t ensure_cluster_attr()
{
    static bool done = false;
    if (done) return cudaSuccess;
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kbest_cluster_kernel<W, MapT, Word, BK>);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kbest_cluster_kernel<W, MapT, Word, BK>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kbest_cluster_kernel<W, MapT, Word, BK>,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) done = true;
    return e;
}

template <int W, typename MapT, typename Word, int BK>
static cudaError_t cluster_config(cudaLaunchConfig_t &cfg, cudaLaunchAttribute &attr, int grid,
                                  int block, size_t smem, int cluster, cudaStream_t st)
{
    cudaError_t e = ensure_cluster_attr<W, MapT, Word, BK>();
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3((unsigned)block, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = (unsigned)cluster;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return e;
}

template <int W, typename MapT, typename Word, int BK>
static cudaError_t launch_cluster_one(const KParams &p, int grid, int block, size_t smem,
                                      int cluster, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr;
    cudaError_t e = cluster_config<W, MapT, Word, BK>(cfg, attr, grid, block, smem, cluster, st);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, kbest_cluster_kernel<W, MapT, Word, BK>, p);
}

template <int W, typename MapT, typename Word, int BK>
static cudaError_t cluster_occupancy_one(int block, size_t smem, int cluster, int *out)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr;
    cudaError_t e = cluster_config<W, MapT, Word, BK>(cfg, attr, cluster, block, smem, cluster,
                                                      nullptr);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveClusters(out, kbest_cluster_kernel<W, MapT, Word, BK>, &cfg);
}

// cluster teams are built for the 8-bit-map classes of 2 and 4 words and the 16-bit-map
// classes of 4, 8 and 16 words
#define FASTGED_CLUSTER_DISPATCH(W_, wide, CALL)                                         \
    do {                                                                                 \
        switch (W_) {                                                                    \
        case 2: return CALL(2, uint8_t, uint64_t);                                       \
        case 4: if (wide) return CALL(4, uint16_t, uint64_t);                            \
                else return CALL(4, uint8_t, uint64_t);                                  \
        case 8: return CALL(8, uint16_t, uint64_t);                                      \
        case 16: return CALL(16, uint16_t, uint64_t);                                    \
        default: return cudaErrorInvalidValue;                                           \
        }                                                                                \
    } while (0)

template <int BK>
cudaError_t launch_kbest_cluster_bk(int W, bool wide, const KParams &p, int grid, int block,
                                    size_t smem, int cluster, cudaStream_t st)
{
#define CALL_CL(w, M, Wd) launch_cluster_one<w, M, Wd, BK>(p, grid, block, smem, cluster, st)
    FASTGED_CLUSTER_DISPATCH(W, wide, CALL_CL);
#undef CALL_CL
}

template <int BK>
cudaError_t kbest_cluster_occupancy_bk(int W, bool wide, int block, size_t smem, int cluster,
                                       int *out)
{
#define CALL_CO(w, M, Wd) cluster_occupancy_one<w, M, Wd, BK>(block, smem, cluster, out)
    FASTGED_CLUSTER_DISPATCH(W, wide, CALL_CO);
#undef CALL_CO
}

template <int BK>
cudaError_t launch_kbest_bk(int W, bool wide_map, bool w32, bool sm, const KParams &p, int grid,
                            int block, size_t smem, cudaStream_t st)
{
#define CALL_LAUNCH(w, M, Wd, S_) launch_one<w, M, Wd, S_, BK>(p, grid, block, smem, st)
    FASTGED_DISPATCH(W, wide_map, w32, sm, CALL_LAUNCH);
#undef CALL_LAUNCH
}

template <int BK>
cudaError_t kbest_occupancy_bk(int W, bool wide_map, bool w32, bool sm, int block, size_t smem,
                               int *out)
{
#define CALL_OCC(w, M, Wd, S_) occupancy_one<w, M, Wd, S_, BK>(block, smem, out)
    FASTGED_DISPATCH(W, wide_map, w32, sm, CALL_OCC);
#undef CALL_OCC
}

}  // namespace fastged
