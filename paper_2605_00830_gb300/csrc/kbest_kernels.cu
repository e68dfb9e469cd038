// kbest_kernels.cu -- sm_103a kernels of the K-Best GED path.
//
//   pack_kernel   S0: edge lists -> adjacency bitsets and edge-label bit-planes
//   kbest_kernel  S1-S5 for every pair of a size class: persistent teams pull pairs from a
//                 device work queue; per level they stage the vertex-cost row, build per-node
//                 neighbour bitsets, score every successor with AND/XOR + popcount, select the
//                 best K with a deterministic stable counting sort, write the kept children in
//                 key order, and finally complete the leaves and take the argmin.
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
// S0: pack edge lists into bitsets (one warp per graph, lanes over its edges).
// ------------------------------------------------------------------------------------
__global__ void pack_kernel(const PackParams pp)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int g = gw; g < pp.n_graphs; g += nwarps) {
        const GraphMeta mt = pp.gmeta[g];
        uint64_t *A = pp.adj + mt.adj_off;
        for (int k = lane; k < mt.m; k += 32) {
            const int64_t e = mt.edge_off + k;
            const int u = pp.edges[2 * e], v = pp.edges[2 * e + 1];
            const unsigned long long bu = 1ull << (u & 63), bv = 1ull << (v & 63);
            const unsigned long long old =
                atomicOr((unsigned long long *)&A[(int64_t)u * mt.W + (v >> 6)], bv);
            if (old & bv) atomicOr(pp.err, kErrDuplicateEdge);
            atomicOr((unsigned long long *)&A[(int64_t)v * mt.W + (u >> 6)], bu);
            if (pp.elabel) {
                const int lab = pp.elabel[e];
                for (int b = 0; b < pp.B; ++b) {
                    if (!((lab >> b) & 1)) continue;
                    uint64_t *Pl = pp.planes + mt.plane_off + (int64_t)b * mt.n * mt.W;
                    atomicOr((unsigned long long *)&Pl[(int64_t)u * mt.W + (v >> 6)], bv);
                    atomicOr((unsigned long long *)&Pl[(int64_t)v * mt.W + (u >> 6)], bu);
                }
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// K-Best teams
// ------------------------------------------------------------------------------------
struct TeamShared {
    int pair;
    int newL;
    int pbase;
    int delcost;
    int cnt;
    int mx;
    int maxb;     // largest histogram bucket touched at this level
    int thr;      // bucket holding the K-th smallest PED
    int wmaxb[kMaxWarps];
    int wn[kMaxWarps];    // candidates each warp scored at this level
    int wlt[kMaxWarps];
    int weq[kMaxWarps];
    unsigned long long wbest[kMaxWarps];
};

template <typename Word>
struct Regions {
    int32_t *hist, *bbase, *alpha2, *sbase, *sel, *selped, *foff, *klist, *kped, *cand;
    int32_t *ped0, *ped1;
    Word *a2t, *l2t, *img0, *img1, *P, *PL;
    uint8_t *map0, *map1, *flist;
};

// A kept child is stored in the selection list as (parent slot << 11) | j, j = 0..n2.
constexpr int kSelShift = 11;

__device__ __forceinline__ int popcw(uint32_t x) { return __popc(x); }
__device__ __forceinline__ int popcw(uint64_t x) { return __popcll(x); }

// mask of lanes <= this lane
__device__ __forceinline__ unsigned lanemask_le() { return 0xffffffffu >> (31 - (threadIdx.x & 31)); }

#ifdef FASTGED_PHASE_TIMERS
// profiling builds only: cycles thread 0 of every team spends in each phase
__device__ unsigned long long g_phase_cycles[8];
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

// Slot owning the candidate stored at index c: the last slot whose first candidate is at
// or before c (first-candidate offsets increase with the slot).
template <typename Word>
__device__ __forceinline__ int slot_of(const Regions<Word> &R, int L, int c)
{
    int lo = 0, hi = L - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (R.foff[mid] <= c) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Stable compaction of the kept successors of this warp, in enumeration order: every
// candidate with PED < T, and the first q with PED == T counted over the whole team.
// keep_before / eq_before: kept / tied candidates of the warps before this one.
template <typename Word>
__device__ __forceinline__ void compact_kept(const Regions<Word> &R, int base, int n, int T,
                                            int q, int keep_before, int eq_before)
{
    const int lane = threadIdx.x & 31;
    for (int kb = 0; kb < n; kb += 32) {
        const int k = kb + lane;
        const int v = k < n ? R.cand[base + k] : INT_MAX;
        if (__ballot_sync(0xffffffffu, v <= T) == 0u) continue;
        const bool is_eq = (v == T);
        const unsigned eqb = __ballot_sync(0xffffffffu, is_eq);
        const int eq_rank = eq_before + __popc(eqb & lanemask_lt());
        const bool keep = (v < T) || (is_eq && eq_rank < q);
        const unsigned kbm = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const int pos = keep_before + __popc(kbm & lanemask_lt());
            R.klist[pos] = base + k;
            R.kped[pos] = v;
        }
        keep_before += __popc(kbm);
        eq_before += __popc(eqb);
    }
}

// Exact selection used when the kept set reaches past the histogram window: the K-th
// smallest PED is found by bisection over team-wide counts, the kept candidates are
// compacted stably, and ranked by (PED, enumeration order).
template <typename MapT, typename Word>
__device__ __noinline__ void select_exact(int32_t *cand, int32_t *klist, int32_t *kped,
                                          const int32_t *foff, const uint8_t *flist_b,
                                          int32_t *sel, int32_t *selped, TeamShared &S, int L,
                                          int stride, int n2, int newL, int lo)
{
    Regions<Word> R;
    R.cand = cand;
    R.klist = klist;
    R.kped = kped;
    R.foff = (int32_t *)foff;
    R.flist = (uint8_t *)flist_b;
    R.sel = sel;
    R.selped = selped;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = blockDim.x, NW = T >> 5;
    const int s_lo = (warp * L) / NW;
    const int base = s_lo * stride, n = S.wn[warp];

    int mx = 0;
    for (int k = lane; k < n; k += 32) mx = max(mx, R.cand[base + k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (tid == 0) S.mx = 0;
    __syncthreads();
    if (lane == 0) atomicMax(&S.mx, mx);
    __syncthreads();
    int hi = S.mx;
    if (lo > hi) lo = hi;
    // invariant: count(PED < lo) < newL <= count(PED <= hi)
    while (lo < hi) {
        const int mid = lo + (hi - lo) / 2;
        int cnt = 0;
        for (int k = lane; k < n; k += 32) cnt += (R.cand[base + k] <= mid);
        cnt = warp_sum(cnt);
        __syncthreads();
        if (tid == 0) S.cnt = 0;
        __syncthreads();
        if (lane == 0) atomicAdd(&S.cnt, cnt);
        __syncthreads();
        if (S.cnt >= newL) hi = mid; else lo = mid + 1;
    }
    const int thr = lo;
    int nlt = 0, neq = 0;
    for (int k = lane; k < n; k += 32) {
        const int v = R.cand[base + k];
        nlt += (v < thr);
        neq += (v == thr);
    }
    nlt = warp_sum(nlt);
    neq = warp_sum(neq);
    if (lane == 0) { S.wlt[warp] = nlt; S.weq[warp] = neq; }
    __syncthreads();
    int lt_all = 0;
    for (int w = 0; w < NW; ++w) lt_all += S.wlt[w];
    const int q = newL - lt_all;
    int keep_before = 0, eq_before = 0;
    for (int w = 0; w < warp; ++w) {
        keep_before += S.wlt[w];
        eq_before += S.weq[w];
    }
    keep_before += min(q, eq_before);
    compact_kept<Word>(R, base, n, thr, q, keep_before, eq_before);
    __syncthreads();
    // rank by (PED, enumeration order); klist is in enumeration order
    for (int a = tid; a < newL; a += T) {
        const int pa = R.kped[a];
        int rank = 0;
        for (int b = 0; b < newL; ++b) {
            const int pb = R.kped[b];
            rank += (pb < pa) || (pb == pa && b < a);
        }
        const int c = R.klist[a];
        const int s = slot_of<Word>(R, L, c);
        const int r = c - R.foff[s];
        const int j = (int)((const MapT *)R.flist)[(int64_t)s * stride + r];
        R.sel[rank] = (s << kSelShift) | j;
        R.selped[rank] = pa;
    }
}

template <int W, typename MapT, typename Word>
__device__ __forceinline__ void solve_pair(const KParams &p, const Regions<Word> R,
                                           TeamShared &S, const int pair)
{
    constexpr int WB = 8 * (int)sizeof(Word);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = blockDim.x, NW = T >> 5;
    const int g1 = p.pairs[2 * pair], g2 = p.pairs[2 * pair + 1];
    const GraphMeta m1 = p.gmeta[g1], m2 = p.gmeta[g2];
    const int n1 = m1.n, n2 = m2.n, W1 = m1.W, W2 = m2.W;
    const int K = p.kpp ? p.kpp[pair] : p.K;
    const int B = p.lay.B;
    const int N2S = p.lay.n2s;
    const int KM = p.lay.kmax;
    const int64_t mrow = p.lay.mrow;
    const int stride = n2 + 1;   // successors of one node: n2 substitutions + the deletion
    const MapT DEL = (MapT)~(MapT)0;
    const CostModel c = p.cost;
    const int hwin = p.hwin;
    const bool fold_ie = (c.eins == c.edel);
    MapT *flist = (MapT *)R.flist;
#ifdef FASTGED_PHASE_TIMERS
    long long ph[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long ph_last = clock64();
#endif

    // stage g2: transposed adjacency and label planes, vertex labels; clear the histogram
    {
        const uint64_t *adj2 = p.adj + m2.adj_off;
        for (int idx = tid; idx < W * n2; idx += T) {
            const int w = idx / n2, u = idx - w * n2;
            const int w64 = (w * WB) >> 6, sh = (w * WB) & 63;
            R.a2t[w * N2S + u] = (w64 < W2) ? (Word)(adj2[(int64_t)u * W2 + w64] >> sh) : (Word)0;
        }
        for (int b = 0; b < B; ++b) {
            const uint64_t *pl2 = p.planes + m2.plane_off + (int64_t)b * n2 * W2;
            for (int idx = tid; idx < W * n2; idx += T) {
                const int w = idx / n2, u = idx - w * n2;
                const int w64 = (w * WB) >> 6, sh = (w * WB) & 63;
                R.l2t[(b * W + w) * N2S + u] =
                    (w64 < W2) ? (Word)(pl2[(int64_t)u * W2 + w64] >> sh) : (Word)0;
            }
        }
        for (int u = tid; u < n2; u += T) R.alpha2[u] = p.vlab[m2.lab_off + u];
        for (int x = tid; x < hwin * NW; x += T) R.hist[x] = 0;
        // root node: empty lambda, R_V2 = V2, PED 0
        for (int w = tid; w < W; w += T) R.img0[w] = (Word)0;
        if (tid == 0) {
            R.ped0[0] = 0;
            S.maxb = -1;
        }
    }
    long long nevals = 0;
    int L = 1;
    // current / next beam buffers, swapped after every level
    uint8_t *mapc = R.map0, *mapn = R.map1;
    Word *imgc = R.img0, *imgn = R.img1;
    int32_t *pedc = R.ped0, *pedn = R.ped1;
    __syncthreads();
    PHASE_MARK(0);

    for (int i = 0; i < n1; ++i) {
        const uint64_t *row1 = p.adj + m1.adj_off + (int64_t)i * W1;
        const uint64_t *pl1 = p.planes + m1.plane_off + (int64_t)i * W1;
        const int64_t pl1_step = (int64_t)n1 * W1;
        const int a1 = p.vlab[m1.lab_off + i];
        int deg = 0;   // neighbours of v_i among v_0..v_{i-1}
        for (int w = lane; w < W1; w += 32) deg += __popcll(row1[w] & low_mask(i, w));
        deg = warp_sum(deg);
        const int delcost = c.vdel + c.edel * deg;   // v_i -> eps takes those edges with it
        const int pbase = pedc[0];                   // the kept list is sorted: slot 0 is least
        const int s_lo = (warp * L) / NW, s_hi = ((warp + 1) * L) / NW;
        const int base = s_lo * stride;              // this warp's candidate storage
        int32_t *hcol = R.hist + warp;
        // clear the buckets of this warp's column that the previous level touched
        for (int b = lane; b <= S.maxb; b += 32) hcol[b * NW] = 0;

        // ---- S1 + S2 per-node vectors, free lists, and S3 evaluation -----------------
        int kw = 0;      // candidates of this warp so far
        int wmaxb = -1;
        for (int g0 = s_lo; g0 < s_hi; g0 += 32) {
            const int ng = min(32, s_hi - g0);
            const int s = g0 + lane;
            const bool act = lane < ng;
            int cnt = 0;
            if (act) {
                // S2: P = images of the substituted g1 neighbours of v_i (and their edge-label
                // planes moved to the image positions); dcnt = deleted neighbours
                Word *Ps = R.P + (int64_t)s * W;
#pragma unroll
                for (int w = 0; w < W; ++w) Ps[w] = (Word)0;
                for (int b = 0; b < B; ++b)
                    for (int w = 0; w < W; ++w) R.PL[((int64_t)b * KM + s) * W + w] = (Word)0;
                const MapT *ms = (const MapT *)(mapc + (int64_t)s * mrow);
                int dcnt = 0;
                for (int w = 0; w < W1; ++w) {
                    uint64_t bits = row1[w] & low_mask(i, w);
                    while (bits) {
                        const int t = __ffsll((long long)bits) - 1;
                        bits &= bits - 1ull;
                        const MapT phi = ms[w * 64 + t];
                        if (phi == DEL) { ++dcnt; continue; }
                        const int pw = (int)phi / WB;
                        const Word pb = (Word)1 << ((int)phi % WB);
                        Ps[pw] |= pb;
                        for (int b = 0; b < B; ++b)
                            if ((pl1[b * pl1_step + w] >> t) & 1ull)
                                R.PL[((int64_t)b * KM + s) * W + pw] |= pb;
                    }
                }
                R.sbase[s] = pedc[s] + c.edel * dcnt;
                const Word *im = imgc + (int64_t)s * W;
                int used = 0;
#pragma unroll
                for (int w = 0; w < W; ++w) used += popcw(im[w]);
                cnt = n2 - used + 1;   // free g2 vertices (R_V2) and the deletion
            }
            // free lists: the free g2 vertices of each slot in increasing order, then n2 for
            // v_i -> eps (lanes over vertices, ballot compaction)
            for (int t = 0; t < ng; ++t) {
                const int st_ = g0 + t;
                const Word *im = imgc + (int64_t)st_ * W;
                MapT *fl = flist + (int64_t)st_ * stride;
                int pos = 0;
                for (int jb = 0; jb < n2; jb += 32) {
                    const int j = jb + lane;
                    const bool fr = j < n2 && !((im[j / WB] >> (j % WB)) & (Word)1);
                    const unsigned bal = __ballot_sync(0xffffffffu, fr);
                    if (fr) fl[pos + __popc(bal & lanemask_lt())] = (MapT)j;
                    pos += __popc(bal);
                }
                if (lane == 0) fl[pos] = (MapT)n2;
            }
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const int excl = incl - cnt;
            const int gtot = __shfl_sync(0xffffffffu, incl, 31);
            if (act) R.foff[s] = base + kw + excl;
            __syncwarp();
            PHASE_MARK(5);

            // S3: lanes walk the group's successors in enumeration order, 32 at a time
            int before = 0;
            for (int kb = 0; kb < gtot; kb += 32) {
                const int k = kb + lane;
                const int d = excl - kb;
                const unsigned bit = (act && d >= 0 && d < 32) ? (1u << d) : 0u;
                const unsigned M = __reduce_or_sync(0xffffffffu, bit);
                const int srel = min(before + __popc(M & lanemask_le()) - 1, 31);
                before += __popc(M);
                const int st = __shfl_sync(0xffffffffu, excl, max(srel, 0));
                int ped = INT_MAX;
                if (k < gtot) {
                    const int sc = g0 + srel;
                    const int j = (int)flist[(int64_t)sc * stride + (k - st)];
                    if (j == n2) {
                        ped = pedc[sc] + delcost;
                    } else {
                        const Word *im = imgc + (int64_t)sc * W;
                        const Word *Ps = R.P + (int64_t)sc * W;
                        int x = 0, y = 0, z = 0;
#pragma unroll
                        for (int w = 0; w < W; ++w) {
                            const Word aw = R.a2t[w * N2S + j];
                            const Word ai = aw & im[w];
                            const Word pw = Ps[w];
                            if (fold_ie) {
                                x += popcw((Word)(ai ^ pw));
                            } else {
                                x += popcw((Word)(ai & ~pw));
                                y += popcw((Word)(pw & ~aw));
                            }
                            if (B > 0) {
                                Word ld = (Word)0;
                                for (int b = 0; b < B; ++b)
                                    ld |= R.PL[((int64_t)b * KM + sc) * W + w] ^
                                          R.l2t[(b * W + w) * N2S + j];
                                z += popcw((Word)(aw & pw & ld));
                            }
                        }
                        const int cv = (R.alpha2[j] != a1) ? c.vsub : 0;   // S1: cost row entry
                        ped = R.sbase[sc] + cv + c.eins * x + c.edel * y + c.esub * z;
                    }
                    R.cand[base + kw + k] = ped;
                }
                int bkt = -1;
                if (ped != INT_MAX) {
                    const int dd = ped - pbase;
                    bkt = dd < hwin - 1 ? dd : hwin - 1;
                    wmaxb = bkt > wmaxb ? bkt : wmaxb;
                }
                const unsigned mm = __match_any_sync(0xffffffffu, bkt);
                if (bkt >= 0 && lane == __ffs(mm) - 1) hcol[bkt * NW] += __popc(mm);
            }
            kw += gtot;
            __syncwarp();
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wmaxb = max(wmaxb, __shfl_xor_sync(0xffffffffu, wmaxb, o));
        if (lane == 0) {
            S.wmaxb[warp] = wmaxb;
            S.wn[warp] = kw;
        }
        __syncthreads();
        PHASE_MARK(1);

        // ---- S4 selection: scan of the (bucket, warp) histogram ---------------------
        int maxb = -1;
        for (int w = 0; w < NW; ++w) maxb = max(maxb, S.wmaxb[w]);
        const int nb = maxb + 1;   // >= 1: every node has a deletion child
        // per bucket, exclusive prefix over warps (segments of NW lanes) and bucket totals
        for (int x = tid; x < ((nb * NW + 31) & ~31); x += T) {
            const int b = x / NW, w = x - b * NW;
            const int v = b < nb ? R.hist[x] : 0;
            int incl = v;
            for (int o = 1; o < NW; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (w >= o) incl += y;
            }
            if (b < nb) {
                R.hist[x] = incl - v;
                if (w == NW - 1) R.bbase[b] = incl;
            }
        }
        __syncthreads();
        if (warp == 0) {
            const int per = (nb + 31) >> 5;
            int loc = 0;
            for (int k = 0; k < per; ++k) {
                const int b = lane * per + k;
                if (b < nb) loc += R.bbase[b];
            }
            int incl = loc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            const int nl = min(K, total);
            int run = incl - loc;
            for (int k = 0; k < per; ++k) {
                const int b = lane * per + k;
                if (b < nb) {
                    const int v = R.bbase[b];
                    R.bbase[b] = run;
                    if (run < nl && run + v >= nl) S.thr = b;   // exactly one bucket crosses
                    run += v;
                }
            }
            if (lane == 0) {
                S.newL = nl;
                S.maxb = maxb;
                nevals += total;
            }
        }
        __syncthreads();
        const int newL = S.newL;
        const int thr = S.thr;
        if (thr < hwin - 1) {
            // kept = every candidate below the threshold bucket and the first q of it, in
            // (PED, parent slot, j) order: position = #(smaller PED) + #(equal PED earlier);
            // hist[b][warp] now holds the bucket-b candidates of the warps before this one
            const int q = newL - R.bbase[thr];
            for (int kb = 0; kb < kw; kb += 32) {
                const int k = kb + lane;
                const int v = k < kw ? R.cand[base + k] - pbase : INT_MAX;
                if (__ballot_sync(0xffffffffu, v <= thr) == 0u) continue;
                const int bkt = v <= thr ? v : -1;
                const unsigned mm = __match_any_sync(0xffffffffu, bkt);
                if (bkt >= 0) {
                    const int rank = hcol[bkt * NW] + __popc(mm & lanemask_lt());
                    if (bkt < thr || rank < q) {
                        const int pos = R.bbase[bkt] + rank;
                        // decode the parent slot and target vertex of candidate base + k
                        int lo = s_lo, hi = s_hi - 1;
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (R.foff[mid] <= base + k) lo = mid; else hi = mid - 1;
                        }
                        const int j = (int)flist[(int64_t)lo * stride + (base + k - R.foff[lo])];
                        R.sel[pos] = (lo << kSelShift) | j;
                        R.selped[pos] = v + pbase;
                    }
                }
                __syncwarp();
                if (bkt >= 0 && lane == __ffs(mm) - 1) hcol[bkt * NW] += __popc(mm);
                __syncwarp();
            }
        } else {
            select_exact<MapT, Word>(R.cand, R.klist, R.kped, R.foff, R.flist, R.sel, R.selped,
                                     S, L, stride, n2, newL, pbase + hwin - 1);
        }
        __syncthreads();
        PHASE_MARK(2);

        // ---- kept children, in key order (slot = rank) -----------------------------
        {
            const int nvec = (int)((i * (int)sizeof(MapT) + 15) >> 4);
            if (mrow <= 128) {
                for (int r = tid; r < newL; r += T) {
                    const int v = R.sel[r];
                    const int s = v >> kSelShift, j = v & ((1 << kSelShift) - 1);
                    const uint4 *src = (const uint4 *)(mapc + (int64_t)s * mrow);
                    uint4 *dst = (uint4 *)(mapn + (int64_t)r * mrow);
                    for (int t = 0; t < nvec; ++t) dst[t] = src[t];
                    ((MapT *)dst)[i] = (j < n2) ? (MapT)j : DEL;
#pragma unroll
                    for (int w = 0; w < W; ++w) {
                        Word x = imgc[(int64_t)s * W + w];
                        if (j < n2 && j / WB == w) x |= (Word)1 << (j % WB);
                        imgn[(int64_t)r * W + w] = x;
                    }
                    pedn[r] = R.selped[r];
                }
            } else {
                for (int r = warp; r < newL; r += NW) {
                    const int v = R.sel[r];
                    const int s = v >> kSelShift, j = v & ((1 << kSelShift) - 1);
                    const uint4 *src = (const uint4 *)(mapc + (int64_t)s * mrow);
                    uint4 *dst = (uint4 *)(mapn + (int64_t)r * mrow);
                    for (int t = lane; t < nvec; t += 32) dst[t] = src[t];
                    for (int w = lane; w < W; w += 32) {
                        Word x = imgc[(int64_t)s * W + w];
                        if (j < n2 && j / WB == w) x |= (Word)1 << (j % WB);
                        imgn[(int64_t)r * W + w] = x;
                    }
                    __syncwarp();
                    if (lane == 0) {
                        ((MapT *)dst)[i] = (j < n2) ? (MapT)j : DEL;
                        pedn[r] = R.selped[r];
                    }
                }
            }
        }
        __syncthreads();
        PHASE_MARK(3);
        { uint8_t *t = mapc; mapc = mapn; mapn = t; }
        { Word *t = imgc; imgc = imgn; imgn = t; }
        { int32_t *t = pedc; pedc = pedn; pedn = t; }
        L = newL;
    }

    // ---- S5 leaf completion (insert the free g2 vertices and their edges) + argmin ------
    {
        unsigned long long best = ~0ull;
        for (int s = warp; s < L; s += NW) {
            const Word *im = imgc + (int64_t)s * W;
            int acc = 0;
            for (int u = lane; u < n2; u += 32) {
                if ((im[u / WB] >> (u % WB)) & (Word)1) {
#pragma unroll
                    for (int w = 0; w < W; ++w) acc += popcw((Word)(R.a2t[w * N2S + u] & im[w]));
                }
            }
            int nimg = 0;
            for (int w = lane; w < W; w += 32) nimg += popcw(im[w]);
            acc = warp_sum(acc);
            nimg = warp_sum(nimg);
            // g2 edges with both ends used were counted twice in acc
            const long long total = (long long)pedc[s] + (long long)c.vins * (n2 - nimg) +
                                    (long long)c.eins * (m2.m - acc / 2);
            const unsigned long long key = ((unsigned long long)total << 32) | (unsigned)s;
            best = key < best ? key : best;
        }
        if (lane == 0) S.wbest[warp] = best;
        __syncthreads();
        if (tid == 0) {
            unsigned long long b = S.wbest[0];
            for (int w = 1; w < NW; ++w) b = S.wbest[w] < b ? S.wbest[w] : b;
            S.wbest[0] = b;
            p.out_cost[pair] = (int32_t)(b >> 32);
            if (p.out_nevals) p.out_nevals[pair] = nevals + L;
        }
        __syncthreads();
        const int bs = (int)(S.wbest[0] & 0xffffffffull);
        const MapT *mb = (const MapT *)(mapc + (int64_t)bs * mrow);
        int32_t *om = p.out_map + p.map_off[pair];
        for (int k = tid; k < n1; k += T) {
            const MapT v = mb[k];
            om[k] = (v == DEL) ? -1 : (int32_t)v;
        }
        __syncthreads();
        PHASE_MARK(4);
    }
#ifdef FASTGED_PHASE_TIMERS
    if (tid == 0)
        for (int k = 0; k < 6; ++k) atomicAdd(&g_phase_cycles[k], (unsigned long long)ph[k]);
#endif
}

// SM: every region lives in shared memory (addresses then stay in the shared window)
template <int W, typename MapT, typename Word, bool SM>
__global__ void __launch_bounds__(512, 2) kbest_kernel(const KParams p)
{
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ TeamShared S;
    uint8_t *gs = p.gscratch + (int64_t)blockIdx.x * p.lay.slice_bytes;
    auto base = [&](int r) -> uint8_t * {
        if (SM) return smem + p.lay.off[r];
        return ((p.lay.smem_mask >> r) & 1u ? smem : gs) + p.lay.off[r];
    };
    Regions<Word> R;
    R.hist = (int32_t *)base(RG_HIST);
    R.bbase = (int32_t *)base(RG_BBASE);
    R.alpha2 = (int32_t *)base(RG_ALPHA2);
    R.a2t = (Word *)base(RG_A2T);
    R.l2t = (Word *)base(RG_L2T);
    R.sbase = (int32_t *)base(RG_SBASE);
    R.ped0 = (int32_t *)base(RG_PED0);
    R.ped1 = (int32_t *)base(RG_PED1);
    R.sel = (int32_t *)base(RG_SEL);
    R.selped = (int32_t *)base(RG_SELPED);
    R.foff = (int32_t *)base(RG_FOFF);
    R.klist = (int32_t *)base(RG_KLIST);
    R.kped = (int32_t *)base(RG_KPED);
    R.img0 = (Word *)base(RG_IMG0);
    R.img1 = (Word *)base(RG_IMG1);
    R.P = (Word *)base(RG_P);
    R.PL = (Word *)base(RG_PL);
    R.flist = base(RG_FLIST);
    R.cand = (int32_t *)base(RG_CAND);
    R.map0 = base(RG_MAP0);
    R.map1 = base(RG_MAP1);

    for (;;) {
        if (threadIdx.x == 0) S.pair = atomicAdd(p.queue_head, 1);
        __syncthreads();
        const int qi = S.pair;
        __syncthreads();
        if (qi >= p.n_order) break;
        solve_pair<W, MapT, Word>(p, R, S, p.order[qi]);
    }
}

// ------------------------------------------------------------------------------------
// launch wrappers (host side of this translation unit)
// ------------------------------------------------------------------------------------
// Opts the kernel into the device's full dynamic shared memory (needed above 48 KB) before
// it is launched or queried for occupancy.
template <int W, typename MapT, typename Word, bool SM>
static cudaError_t ensure_smem_attr()
{
    static bool done = false;
    if (done) return cudaSuccess;
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kbest_kernel<W, MapT, Word, SM>);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kbest_kernel<W, MapT, Word, SM>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) done = true;
    return e;
}

template <int W, typename MapT, typename Word, bool SM>
static cudaError_t launch_one(const KParams &p, int grid, int block, size_t smem,
                              cudaStream_t st)
{
    cudaError_t e = ensure_smem_attr<W, MapT, Word, SM>();
    if (e != cudaSuccess) return e;
    kbest_kernel<W, MapT, Word, SM><<<grid, block, smem, st>>>(p);
    return cudaGetLastError();
}

template <int W, typename MapT, typename Word, bool SM>
static cudaError_t occupancy_one(int block, size_t smem, int *out)
{
    cudaError_t e = ensure_smem_attr<W, MapT, Word, SM>();
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, kbest_kernel<W, MapT, Word, SM>,
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

bool kbest_has_smem_variant(int W, bool wide, bool w32) { return w32 || (W <= 4 && !wide); }

cudaError_t launch_kbest(int W, bool wide_map, bool w32, bool sm, const KParams &p, int grid,
                         int block, size_t smem, cudaStream_t st)
{
#define CALL_LAUNCH(w, M, Wd, S_) launch_one<w, M, Wd, S_>(p, grid, block, smem, st)
    FASTGED_DISPATCH(W, wide_map, w32, sm, CALL_LAUNCH);
#undef CALL_LAUNCH
}

cudaError_t kbest_occupancy(int W, bool wide_map, bool w32, bool sm, int block, size_t smem,
                            int *out)
{
#define CALL_OCC(w, M, Wd, S_) occupancy_one<w, M, Wd, S_>(block, smem, out)
    FASTGED_DISPATCH(W, wide_map, w32, sm, CALL_OCC);
#undef CALL_OCC
}

cudaError_t launch_pack(const PackParams &pp, int n_graphs, cudaStream_t st)
{
    const int block = 256;
    int grid = (n_graphs * 32 + block - 1) / block;
    if (grid < 1) grid = 1;
    if (grid > 4096) grid = 4096;
    pack_kernel<<<grid, block, 0, st>>>(pp);
    return cudaGetLastError();
}

// upper bound of the kernels' static shared memory (the team's scalars)
size_t team_shared_static_bytes() { return sizeof(TeamShared) + 256; }

}  // namespace fastged

#ifdef FASTGED_PHASE_TIMERS
// profiling builds only: reads (and optionally clears) the per-phase cycle counters
extern "C" int fastged_debug_phase_cycles(unsigned long long *out, int reset)
{
    if (cudaMemcpyFromSymbol(out, fastged::g_phase_cycles, sizeof(unsigned long long) * 8) !=
        cudaSuccess)
        return -3;
    if (reset) {
        unsigned long long z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        cudaMemcpyToSymbol(fastged::g_phase_cycles, z, sizeof(z));
    }
    return 0;
}
#endif
