// kbest_warp.cuh -- sm_103a K-Best kernel with one warp per pair, for pairs whose target graph
// fits one bitset word with a bit to spare (n2 <= 63; the bit after the last vertex stands for
// the deletion), whose source has at most 64 vertices and whose beam is small (the
// molecule-like batches). Instantiated per edge-label plane count in kbest_b0.cu,
// kbest_b2.cu and kbest_b8.cu next to the team kernels of kbest_impl.cuh.
//
// Method: Algorithm 1 of Dabah & Herten (branching Sec. 4.1.1, evaluation Sec. 4.1.2 and
// Algorithm 2, selection Sec. 4.2, leaf insertions Sec. 4.4), with the bitset form of the
// implied edge costs stated at the top of kbest_impl.cuh. Results are identical to the team
// kernels' (same key order, same tie-breaking); only the mapping onto the hardware differs:
//
//   * a warp owns a pair, so a level needs no block barrier and no cross-warp table;
//   * evaluation runs lane <-> parent node: each lane keeps its node's vectors (Img, P, label
//     planes of P, base PED) in registers and walks the node's successor bitset (its free
//     target vertices, and the deletion as bit n2) in increasing order, so no successor-id
//     list is built; every step of that walk scores one successor per lane against the
//     staged target record of its bit, without branches. A group of at most 16 nodes (the
//     tail of the beam, or an early level) gives each node 2-32 lanes, each walking one
//     slice of the bit range 0..n2;
//   * the PED histogram of the selection is counted in the same loop in per-lane 4-bit
//     counters (offsets 0-14 from the anchor, widened to 16 bits every 14 slots and summed
//     over the warp once per level), anchored at the PED of the best parent, a lower bound of
//     every child (costs are non-negative and slot 0 holds the least PED of the kept list).
//     Costs are scaled by 4 inside the evaluation, so that an offset is the bit position of
//     its counter; the slots past a lane's successors score a stand-in record whose offset
//     is past every bucket;
//   * each successor leaves one 16-bit entry (PED offset clamped to 8 bits, record index) in
//     enumeration order (node by node, j increasing, the deletion last); the kept ones are
//     compacted in that order and then placed at their rank by a counting sort over the
//     buckets;
//   * when the K-th PED falls past the histogram window, the level is scored again with exact
//     16-bit PED offsets (every PED of a pair routed here is below 2^16), the K-th offset is
//     found by bisection, the kept entries are ranked by (PED, enumeration order) and their
//     target vertices recovered from the node's free set.
#pragma once
#include "kbest_impl.cuh"

namespace fastged {

// x << n with PTX semantics: shift amounts of 32 or more give 0
__device__ __forceinline__ uint32_t shl_clamped(uint32_t x, uint32_t n)
{
    uint32_t r;
    asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(n));
    return r;
}

// PED histogram buckets of the one-warp kernel: offsets 0..kWarpBuckets-2 from the anchor
// decide the threshold (the last field of the counters is not read)
constexpr int kWarpBuckets = 16;
// kept successors a warp places at once: the largest K of a one-warp class, in 32s
constexpr int kWarpChunks = 4;
// cost entry of record 0 in quarter units: any slot scoring it has an offset far past every
// histogram bucket, and adding it to a PED offset (below 2^18 in quarter units) stays in range
constexpr int kWarpIdleCost = 1 << 24;

// Target record of g2 vertex u, stored at index u + 1, or of the deletion column, stored at
// index n2 + 1 (no neighbours, no labels): adjacency word, NPL edge-label planes, and the
// vertex-cost entry C[i][u] of the current level times 4 (the evaluation works in units of a
// quarter, so that a PED offset is directly the bit position of its histogram counter).
// Record 0 is a stand-in scored by the slots past a lane's successors: its cost entry is so
// large that such a slot counts in no histogram bucket.
template <typename Word, int NPL>
struct __align__(16) TgtRec {
    Word a2;
    Word l[NPL];
    int32_t crow;
};
template <typename Word>
struct __align__(16) TgtRec<Word, 0> {
    Word a2;
    int32_t crow;
};

static_assert(sizeof(TgtRec<uint32_t, 0>) == warp_rec_bytes(true, 0), "record size");
static_assert(sizeof(TgtRec<uint32_t, 2>) == warp_rec_bytes(true, 2), "record size");
static_assert(sizeof(TgtRec<uint32_t, kMaxB>) == warp_rec_bytes(true, kMaxB), "record size");
static_assert(sizeof(TgtRec<uint64_t, 0>) == warp_rec_bytes(false, 0), "record size");
static_assert(sizeof(TgtRec<uint64_t, 2>) == warp_rec_bytes(false, 2), "record size");
static_assert(sizeof(TgtRec<uint64_t, kMaxB>) == warp_rec_bytes(false, kMaxB), "record size");

template <typename Word, int NPL>
__device__ __forceinline__ Word rec_plane(const TgtRec<Word, NPL> &r, int b) { return r.l[b]; }
template <typename Word>
__device__ __forceinline__ Word rec_plane(const TgtRec<Word, 0> &, int) { return (Word)0; }
template <typename Word, int NPL>
__device__ __forceinline__ void rec_set_plane(TgtRec<Word, NPL> &r, int b, Word v) { r.l[b] = v; }
template <typename Word>
__device__ __forceinline__ void rec_set_plane(TgtRec<Word, 0> &, int, Word) {}

#ifdef FASTGED_PHASE_TIMERS
// profiling builds only: cycles lane 0 of every warp spends in each phase
#define WPHASE(k)                                            \
    do {                                                     \
        if ((threadIdx.x & 31) == 0) {                       \
            const long long t_ = clock64();                  \
            ph[k] += t_ - ph_last;                           \
            ph_last = t_;                                    \
        }                                                    \
    } while (0)
#else
#define WPHASE(k) do { } while (0)
#endif

// 1 + index of the lowest set bit, 0 when none is set: the record index of the next
// successor of a walk (a free target vertex, or the deletion as bit n2), record 0 once the
// walk is over
__device__ __forceinline__ int ffs1(uint32_t x) { return __ffs((int)x); }
__device__ __forceinline__ int ffs1(uint64_t x) { return __ffsll((long long)x); }

// Dynamic shared memory of the one-warp kernel (every warp of a CTA has its block in it).
extern __shared__ __align__(16) uint8_t g_warp_smem[];

// Working set of one warp (see WarpRegion): the warp's block is addressed by 32-bit offsets
// into shared memory; only the vertex maps (shared or global) need full pointers. The beam
// buffers alternate: cur selects which of each pair holds the current level.
template <typename Word, int NPL>
struct WarpRegs {
    uint32_t wb;     // start of the warp's block in dynamic shared memory
    int cur;         // 0: buffers *0 are current, *1 next; 1: the reverse
    uint8_t *mb;     // base of the vertex-map buffers
    template <typename T>
    __device__ __forceinline__ T *at(int32_t off) const { return (T *)(g_warp_smem + wb + (uint32_t)off); }
    __device__ __forceinline__ TgtRec<Word, NPL> *tgt(const WarpLayout &wl) const { return at<TgtRec<Word, NPL>>(wl.off[WR_TGT]); }
    __device__ __forceinline__ int32_t *lab2(const WarpLayout &wl) const { return at<int32_t>(wl.off[WR_LAB2]); }
    __device__ __forceinline__ int32_t *noff(const WarpLayout &wl) const { return at<int32_t>(wl.off[WR_NOFF]); }
    __device__ __forceinline__ int32_t *nbr(const WarpLayout &wl) const { return at<int32_t>(wl.off[WR_NBR]); }
    __device__ __forceinline__ Word *imgc(const WarpLayout &wl) const { return at<Word>(cur ? wl.off[WR_IMG1] : wl.off[WR_IMG0]); }
    __device__ __forceinline__ Word *imgn(const WarpLayout &wl) const { return at<Word>(cur ? wl.off[WR_IMG0] : wl.off[WR_IMG1]); }
    __device__ __forceinline__ int32_t *pedc(const WarpLayout &wl) const { return at<int32_t>(cur ? wl.off[WR_PED1] : wl.off[WR_PED0]); }
    __device__ __forceinline__ int32_t *pedn(const WarpLayout &wl) const { return at<int32_t>(cur ? wl.off[WR_PED0] : wl.off[WR_PED1]); }
    __device__ __forceinline__ uint16_t *e2c(const WarpLayout &wl) const { return at<uint16_t>(cur ? wl.off[WR_E21] : wl.off[WR_E20]); }
    __device__ __forceinline__ uint16_t *e2n(const WarpLayout &wl) const { return at<uint16_t>(cur ? wl.off[WR_E20] : wl.off[WR_E21]); }
    __device__ __forceinline__ uint16_t *ent(const WarpLayout &wl) const { return at<uint16_t>(wl.off[WR_ENT]); }
    __device__ __forceinline__ uint16_t *nodeoff(const WarpLayout &wl) const { return at<uint16_t>(wl.off[WR_NODEOFF]); }
    __device__ __forceinline__ uint32_t *klist(const WarpLayout &wl) const { return at<uint32_t>(wl.off[WR_KLIST]); }
    __device__ __forceinline__ int32_t *sel(const WarpLayout &wl) const { return at<int32_t>(wl.off[WR_SEL]); }
    __device__ __forceinline__ int32_t *selped(const WarpLayout &wl) const { return at<int32_t>(wl.off[WR_SELPED]); }
    __device__ __forceinline__ uint8_t *mapc(const WarpLayout &wl) const { return mb + (cur ? wl.off[WR_MAP1] : wl.off[WR_MAP0]); }
    __device__ __forceinline__ uint8_t *mapn(const WarpLayout &wl) const { return mb + (cur ? wl.off[WR_MAP0] : wl.off[WR_MAP1]); }
};

// Scores every successor of level i (lane <-> parent node). Entries go to ent in enumeration
// order and nodeoff receives each node's first entry. EXACT = false: entry = (min(PED - A,
// 255) << 8) | (record index: 1 + target vertex, n2 + 1 for the deletion), and on return lane
// b < kWarpBuckets - 1 holds the number of successors whose offset PED - A is b (lane
// kWarpBuckets - 1 holds no meaningful count); EXACT = true: entry = PED - A (exact, below
// 2^16).
// FOLD: insertion and deletion of an edge cost the same, so the two implied-edge terms are
// one popcount. Returns the number of successors of the level.
template <typename Word, int BK, bool FOLD, bool EXACT>
__device__ __forceinline__ int eval_level(const KParams &p,
                                          const WarpRegs<Word, (BK == 8 ? kMaxB : BK)> &R,
                                          int L, int n0, int deg, int n2, int mrow, int A,
                                          int &hist, long long *prof = nullptr)
{
    constexpr int WB = 8 * (int)sizeof(Word);
    constexpr int NPL = BK == 8 ? kMaxB : BK;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const WarpLayout &wl = p.wl;
    const int B = BK == 0 ? 0 : (BK == 2 ? 2 : p.lay.B);
    // costs in quarter units (see TgtRec): a successor's PED offset times 4 is the bit
    // position of its 4-bit histogram counter in the 64-bit pair (chi, clo)
    const int c_eins = 4 * p.cost.eins, c_edel = 4 * p.cost.edel, c_esub = 4 * p.cost.esub;
    const Word nmask = n2 >= WB ? ~(Word)0 : (((Word)1 << n2) - (Word)1);
    const uint8_t *mapc = R.mapc(wl);
    using TRec = TgtRec<Word, NPL>;
    const TRec *tgt = R.tgt(wl);
    // histogram: 4-bit counters (clo: buckets 0-7, chi: 8-15) widened every 14 slots into
    // acc[m] = buckets (m, m + 4) and acc[4 + m] = (8 + m, 12 + m), 16 bits each
    uint32_t clo = 0, chi = 0, acc[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) acc[m] = 0;
    auto flush = [&]() {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            acc[m] += (clo >> (4 * m)) & 0x000F000Fu;
            acc[4 + m] += (chi >> (4 * m)) & 0x000F000Fu;
        }
        clo = chi = 0;
    };
    int tot = 0;
    // v_i's first prior neighbour (the same for every node): most levels of tree-like source
    // graphs have at most one, and those take the short S2 path below
    const int e0 = deg > 0 ? FG_AT(R.nbr(wl), n0, FG_N(int32_t, wl.size[WR_NBR])) : -1;
#ifdef FASTGED_PHASE_TIMERS
    long long tprof = clock64();
#endif
    for (int g0 = 0; g0 < L; g0 += 32) {
        // a group of ng nodes: one lane per node when ng > 16, else q = 2^qs lanes per node
        // (ng * q <= 32), lane part r taking the successors in its slice of the bit range
        // 0..n2 (target vertices, then the deletion as bit n2), so that a short group (the
        // last of a beam of 100, or a level of few nodes) keeps every lane busy
        const int ng = min(32, L - g0);
        const int qs = ng > 16 ? 0 : ng > 8 ? 1 : ng > 4 ? 2 : ng > 2 ? 3 : ng > 1 ? 4 : 5;
        const int q = 1 << qs;
        const int r = lane & (q - 1);
        const int s = g0 + (lane >> qs);
        const bool act = (lane >> qs) < ng;
        // S2: P = images of the substituted g1 neighbours of v_i, their edge labels as planes
        // at the image positions, dcnt = deleted neighbours (the neighbour list is the same
        // for every lane: v_i's prior neighbours)
        Word P = (Word)0;
        Word PL[NPL > 0 ? NPL : 1];
#pragma unroll
        for (int b = 0; b < (NPL > 0 ? NPL : 1); ++b) PL[b] = (Word)0;
        int dcnt = 0;
        const int64_t ms = (int64_t)(act ? s : 0) * mrow;   // the node's map row
        if (deg <= 1) {   // warp-uniform
            if (deg == 1) {
                const uint8_t ph = act ? FG_AT(mapc, ms + (e0 & 0xffff), wl.size[WR_MAP0]) : (uint8_t)0xff;
                const bool sub = ph != 0xff;
                dcnt = sub ? 0 : 1;
                P = sub ? (Word)1 << ph : (Word)0;
#pragma unroll
                for (int b = 0; b < NPL; ++b)
                    if (b < B && ((e0 >> (16 + b)) & 1)) PL[b] = P;
            }
        } else
        for (int t0 = 0; t0 < deg; t0 += 4) {
            int e[4];
            uint8_t phi[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                e[u] = t0 + u < deg ? FG_AT(R.nbr(wl), n0 + t0 + u, FG_N(int32_t, wl.size[WR_NBR])) : -1;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                phi[u] = (e[u] >= 0 && act) ? FG_AT(mapc, ms + (e[u] & 0xffff), wl.size[WR_MAP0])
                                            : (uint8_t)0xff;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool sub = phi[u] != 0xff;
                dcnt += (e[u] >= 0 && !sub) ? 1 : 0;
                const Word pb = sub ? (Word)1 << phi[u] : (Word)0;
                P |= pb;
#pragma unroll
                for (int b = 0; b < NPL; ++b)
                    if (b < B && ((e[u] >> (16 + b)) & 1)) PL[b] |= pb;
            }
        }
        const Word im = act ? FG_AT(R.imgc(wl), s, FG_N(Word, wl.size[WR_IMG0])) : ~(Word)0;
        const int base = act ? 4 * (FG_AT(R.pedc(wl), s, FG_N(int32_t, wl.size[WR_PED0])) - A) + c_edel * dcnt
                             : 0;
        // the node's successors: its free target vertices and the deletion as bit n2 (n2 < WB)
        const Word fr = act ? (Word)((~im & nmask) | ((Word)1 << n2)) : (Word)0;
        const int ncnt = popcw(fr);
        // this lane's slice [lo, hi) of the bits 0..n2 (hi <= n2 + 1 <= WB)
        const int lo = (r * (n2 + 1)) >> qs, hi = ((r + 1) * (n2 + 1)) >> qs;
        const Word below = lo >= WB ? ~(Word)0 : (((Word)1 << lo) - (Word)1);
        const Word upto = hi >= WB ? ~(Word)0 : (((Word)1 << hi) - (Word)1);
        Word x = fr & upto & ~below;
        const int cnt = popcw(x);   // this lane's successors
        int incl = r == 0 ? ncnt : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        const int noff = tot + incl - ncnt;   // the node's first entry (same on all its parts)
        if (act && r == 0) FG_AT(R.nodeoff(wl), s, FG_N(uint16_t, wl.size[WR_NODEOFF])) = (uint16_t)noff;
        const int off = noff + popcw((Word)(fr & below));   // this lane's first entry
        const int maxc = (int)__reduce_max_sync(FULL, (unsigned)cnt);
#ifdef FASTGED_PHASE_TIMERS
        // profiling builds: loop slots of the level, cycles of the group set-up (prof[12])
        if (prof && lane == 0) {
            const long long tn = clock64();
            prof[9] += maxc;
            prof[12] += tn - tprof;
            tprof = tn;
        }
#endif
        uint16_t *ent = R.ent(wl);
        // two successors of the lane's slice per step (its next two bits, or record 0 once
        // none is left), in blocks of 14 so that a 4-bit counter cannot overflow inside one.
        // score(j) is 4 * (PED - A) of the successor with record j.
        auto score = [&](int j) -> int {
            const TgtRec<Word, NPL> r = FG_AT(tgt, j, FG_N(TRec, wl.size[WR_TGT]));
            const Word ai = r.a2 & im;
            int d = base + r.crow;
            if (FOLD) {
                d += c_eins * popcw((Word)(ai ^ P));
            } else {
                d += c_eins * popcw((Word)(ai & ~P)) + c_edel * popcw((Word)(P & ~r.a2));
            }
            if (NPL > 0) {
                Word ld = (Word)0;
#pragma unroll
                for (int b = 0; b < NPL; ++b)
                    if (b < B) ld |= PL[b] ^ rec_plane(r, b);
                d += c_esub * popcw((Word)(r.a2 & P & ld));
            }
            return d;
        };
        // the 4-bit field of offset d = d4 / 4 starts at bit d4 of the 64-bit pair (chi,
        // clo); a PTX shift by 32 or more yields 0, so the word that does not hold the field
        // gets nothing, and neither does an offset of 16 or more, without a compare. Every
        // slot is counted: the ones past the lane's successors score record 0, whose offset
        // is past every bucket.
        auto count = [&](int d4) {
            clo += shl_clamped(1u, (uint32_t)d4);
            chi += shl_clamped(1u, (uint32_t)d4 - 32u);
        };
        for (int t0 = 0; t0 < maxc; t0 += 14) {
            const int t1 = min(maxc, t0 + 14);
            for (int t = t0; t < t1; t += 2) {
                const int ja = ffs1(x);
                x &= x - (Word)1;
                const int jb = ffs1(x);
                x &= x - (Word)1;
                const bool va = t < cnt, vb = t + 1 < cnt;
                const int da = score(ja), db = score(jb);
#define NE FG_N(uint16_t, wl.size[WR_ENT])
                // predicated stores: the slots past the lane's successors write nothing
                if (EXACT) {
                    if (va) FG_AT(ent, off + t, NE) = (uint16_t)(da >> 2);
                    if (vb) FG_AT(ent, off + t + 1, NE) = (uint16_t)(db >> 2);
                } else {
                    if (va) FG_AT(ent, off + t, NE) = (uint16_t)((min(da, 1020) << 6) | ja);
                    if (vb) FG_AT(ent, off + t + 1, NE) = (uint16_t)((min(db, 1020) << 6) | jb);
#undef NE
                    count(da);
                    count(db);
                }
            }
            if (!EXACT) flush();
        }
#ifdef FASTGED_PHASE_TIMERS
        // profiling builds: cycles of the scoring loop (prof[13])
        if (prof && lane == 0) {
            const long long tn = clock64();
            prof[13] += tn - tprof;
            tprof = tn;
        }
#endif
        tot += __shfl_sync(FULL, incl, 31);
    }
    if (lane == 0) FG_AT(R.nodeoff(wl), L, FG_N(uint16_t, wl.size[WR_NODEOFF])) = (uint16_t)tot;
    if (!EXACT) {
        // warp totals (at most 128 x 65 successors: 16-bit fields cannot overflow), then lane
        // b takes bucket b
#pragma unroll
        for (int m = 0; m < 8; ++m) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[m] += __shfl_xor_sync(FULL, acc[m], o);
        }
        const int b = lane & 15;
        const int wsel = ((b >> 3) << 2) | (b & 3);
        uint32_t wv = acc[0];
#pragma unroll
        for (int m = 1; m < 8; ++m) wv = wsel == m ? acc[m] : wv;
        hist = (int)((wv >> (((b >> 2) & 1) << 4)) & 0xffffu);
    }
    __syncwarp();
#ifdef FASTGED_PHASE_TIMERS
    // profiling builds: cycles after the scoring loops (group tails, warp reduction; prof[14])
    if (prof && lane == 0) prof[14] += clock64() - tprof;
#endif
    return tot;
}

// Slot of the node that owns entry k (nodeoff is strictly increasing: every node has at
// least its deletion successor).
__device__ __forceinline__ int node_of(const KParams &p, const uint16_t *nodeoff, int L, int k)
{
    int lo = 0, hi = L;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;   // 0 < mid < L: within the node offsets
        if ((int)FG_AT(nodeoff, mid, FG_N(uint16_t, p.wl.size[WR_NODEOFF])) <= k) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <typename Word, int BK, bool FOLD>
__device__ __forceinline__ void solve_pair_warp(const KParams &p, uint32_t wb, uint8_t *gw,
                                                const int pair)
{
    constexpr int NPL = BK == 8 ? kMaxB : BK;
    constexpr int WB = 8 * (int)sizeof(Word);
    using Rec = TgtRec<Word, NPL>;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const WarpLayout &wl = p.wl;
    WarpRegs<Word, NPL> R;
    R.wb = wb;
    R.cur = 0;
    R.mb = wl.gmap ? gw : g_warp_smem + wb;

// elements of warp region r viewed as type T (bounds-checked builds check indexes against it)
#define WN(T, r) FG_N(T, wl.size[r])
    const int g1 = FG_AT(p.pairs, 2 * pair, 2 * p.n_pairs);
    const int g2 = FG_AT(p.pairs, 2 * pair + 1, 2 * p.n_pairs);
    const GraphMeta m1 = FG_AT(p.gmeta, g1, p.n_graphs), m2 = FG_AT(p.gmeta, g2, p.n_graphs);
    const int n1 = m1.n, n2 = m2.n, W1 = m1.W;
    const int K = p.kpp ? FG_AT(p.kpp, pair, p.n_pairs) : p.K;
    const int B = BK == 0 ? 0 : (BK == 2 ? 2 : p.lay.B);
    const int mrow = wl.mrow;
    const CostModel c = p.cost;
    // buckets 0..H-2 hold one PED offset each; a K-th offset past them takes the exact fallback
    const int H = min(p.hwin, kWarpBuckets);
    constexpr uint8_t DEL = 0xff;
    // m &= ballot(bit b of an offset) ^ lb[b] keeps the lanes whose bit b equals bit b of
    // this lane's index
    unsigned lb[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) lb[k] = ((lane >> k) & 1) ? 0u : 0xffffffffu;
#ifdef FASTGED_PHASE_TIMERS
    long long ph[16] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    long long ph_last = clock64();
#endif

    // ---- stage the target graph (record u + 1 target vertex u, record n2 + 1 the deletion,
    // record 0 the stand-in of finished walks) and the source graph's prior-neighbour lists
    {
        const uint64_t *adj2 = p.adj + m2.adj_off;
        const uint64_t *pl2 = p.planes + m2.plane_off;
        const int W2 = m2.W;
        for (int k = lane; k <= n2 + 1; k += 32) {
            const int u = k - 1;
            const bool vtx = u >= 0 && u < n2;
            Rec r;
            r.a2 = vtx ? (Word)FG_AT(adj2, (int64_t)u * W2, p.adj_words - m2.adj_off) : (Word)0;
#pragma unroll
            for (int b = 0; b < NPL; ++b)
                rec_set_plane(r, b, (vtx && b < B)
                                        ? (Word)FG_AT(pl2, ((int64_t)b * n2 + u) * W2,
                                                      p.plane_words - m2.plane_off)
                                        : (Word)0);
            r.crow = k == 0 ? kWarpIdleCost : 0;
            FG_AT(R.tgt(wl), k, WN(Rec, WR_TGT)) = r;
            if (vtx)
                FG_AT(R.lab2(wl), u, WN(int32_t, WR_LAB2)) =
                    FG_AT(p.vlab, m2.lab_off + u, p.n_vlab);
        }
        // prior neighbours v_k (k < v) of every g1 vertex v, with their edge labels
        for (int v = lane; v < n1; v += 32) {
            const int64_t row = m1.adj_off + (int64_t)v * W1;
            int d = 0;
            for (int w = 0; w < W1; ++w)
                d += __popcll(FG_AT(p.adj, row + w, p.adj_words) & low_mask(v, w));
            FG_AT(R.noff(wl), v + 1, WN(int32_t, WR_NOFF)) = d;
        }
        __syncwarp();
        int carry = 0;
        for (int v0 = 0; v0 < n1; v0 += 32) {
            const int v = v0 + lane;
            const int d = v < n1 ? FG_AT(R.noff(wl), v + 1, WN(int32_t, WR_NOFF)) : 0;
            int incl = d;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += y;
            }
            __syncwarp();
            if (v < n1) FG_AT(R.noff(wl), v + 1, WN(int32_t, WR_NOFF)) = carry + incl;
            carry += __shfl_sync(FULL, incl, 31);
        }
        if (lane == 0) FG_AT(R.noff(wl), 0, WN(int32_t, WR_NOFF)) = 0;
        __syncwarp();
        const int64_t pstep = (int64_t)n1 * W1;
        for (int v = lane; v < n1; v += 32) {
            const int64_t row = m1.adj_off + (int64_t)v * W1;
            const int64_t pl = m1.plane_off + (int64_t)v * W1;
            int o = FG_AT(R.noff(wl), v, WN(int32_t, WR_NOFF));
            for (int w = 0; w < W1; ++w) {
                uint64_t bits = FG_AT(p.adj, row + w, p.adj_words) & low_mask(v, w);
                while (bits) {
                    const int t = __ffsll((long long)bits) - 1;
                    bits &= bits - 1ull;
                    int lab = 0;
                    for (int b = 0; b < B; ++b)
                        lab |= (int)((FG_AT(p.planes, pl + b * pstep + w, p.plane_words) >> t) & 1ull) << b;
                    FG_AT(R.nbr(wl), o, WN(int32_t, WR_NBR)) = (w * 64 + t) | (lab << 16);
                    ++o;
                }
            }
        }
        // root: empty map, Img empty, PED 0
        if (lane == 0) {
            FG_AT(R.imgc(wl), 0, WN(Word, WR_IMG0)) = (Word)0;
            FG_AT(R.pedc(wl), 0, WN(int32_t, WR_PED0)) = 0;
            FG_AT(R.e2c(wl), 0, WN(uint16_t, WR_E20)) = 0;
        }
        __syncwarp();
    }

    long long nevals = 0;
    int L = 1;
    WPHASE(0);
    for (int i = 0; i < n1; ++i) {
        // S1: this level's vertex-cost row C[i][u] in quarter units (record n2 + 1, the
        // deletion column, holds c_vdel; record 0 keeps its stand-in cost)
        {
            const int a1 = FG_AT(p.vlab, m1.lab_off + i, p.n_vlab);
            for (int k = lane + 1; k <= n2 + 1; k += 32)
                FG_AT(R.tgt(wl), k, WN(Rec, WR_TGT)).crow =
                    4 * (k <= n2 ? ((FG_AT(R.lab2(wl), k - 1, WN(int32_t, WR_LAB2)) != a1) ? c.vsub : 0)
                                 : c.vdel);
        }
        __syncwarp();
        WPHASE(7);
        const int n0 = FG_AT(R.noff(wl), i, WN(int32_t, WR_NOFF));
        const int deg = FG_AT(R.noff(wl), i + 1, WN(int32_t, WR_NOFF)) - n0;
        const int A = FG_AT(R.pedc(wl), 0, WN(int32_t, WR_PED0));   // least PED of the kept list: a lower bound of every child
        int hist = 0;
#ifdef FASTGED_PHASE_TIMERS
        const int tot = eval_level<Word, BK, FOLD, false>(p, R, L, n0, deg, n2, mrow, A, hist,
                                                          ph);
        ph[10] += tot;   // successors (the loop steps above cover them 32 lanes at a time)
        ph[11] += 1;     // levels
#else
        const int tot = eval_level<Word, BK, FOLD, false>(p, R, L, n0, deg, n2, mrow, A, hist);
#endif
        nevals += tot;
        WPHASE(1);
        const int newL = min(K, tot);
        // S4: bucket b = PED - A for b < H - 1; a K-th offset past them goes to the exact
        // fallback
        const int cb = lane < H - 1 ? hist : 0;
        int incl = cb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        const int bexcl = incl - cb;
        const unsigned hb = __ballot_sync(FULL, lane < H - 1 && incl >= newL);
        if (hb) {
            const int thr = __ffs(hb) - 1;
            // kept: every successor below bucket thr and the first q of bucket thr, compacted
            // in enumeration order (the loop stops once all are found)
            const int q = newL - __shfl_sync(FULL, bexcl, thr);
            const int lim = (thr + 1) << 8;   // entry < lim <=> PED offset <= thr
            int keep_before = 0, eq_before = 0;
            for (int kb = 0; kb < tot && keep_before < newL; kb += 128) {
                int e[4];
                unsigned le[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = kb + 32 * u + lane;
                    e[u] = k < tot ? (int)FG_AT(R.ent(wl), k, WN(uint16_t, WR_ENT)) : 0xffff;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) le[u] = __ballot_sync(FULL, e[u] < lim);
                if ((le[0] | le[1] | le[2] | le[3]) == 0u) continue;
                // the four sub-chunks' ties, then their kept sets, each set of ballots taken
                // together (the counts of the sub-chunks before are prefix sums)
                const unsigned lt = lanemask_lt();
                unsigned eqb[4], kbm[4];
                bool keep[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) eqb[u] = __ballot_sync(FULL, (e[u] >> 8) == thr);
                int eqp = eq_before;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int d = e[u] >> 8;
                    keep[u] = (d < thr) || (d == thr && eqp + __popc(eqb[u] & lt) < q);
                    eqp += __popc(eqb[u]);
                }
                eq_before = eqp;
#pragma unroll
                for (int u = 0; u < 4; ++u) kbm[u] = __ballot_sync(FULL, keep[u]);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (keep[u])
                        FG_AT(R.klist(wl), keep_before + __popc(kbm[u] & lt), WN(uint32_t, WR_KLIST)) =
                            ((uint32_t)e[u] << 16) | (uint32_t)(kb + 32 * u + lane);
                    keep_before += __popc(kbm[u]);
                }
            }
            __syncwarp();
            WPHASE(3);
            // place every kept successor at its rank: (smaller offsets) + (equal offsets
            // earlier in enumeration order). All chunks of the kept list are handled at once;
            // lane b carries the kept successors of bucket b in the chunks before each one.
            // A kept entry is its 16-bit successor entry (offset << 8 | record index) << 16 |
            // its index k in enumeration order.
            uint32_t kv[kWarpChunks];
            int dk[kWarpChunks], pos[kWarpChunks];
            bool vk[kWarpChunks];
            int run = 0;
#pragma unroll
            for (int ch = 0; ch < kWarpChunks; ++ch) {
                const int x = 32 * ch + lane;
                vk[ch] = x < newL;
                kv[ch] = vk[ch] ? FG_AT(R.klist(wl), x, WN(uint32_t, WR_KLIST)) : 0u;
                dk[ch] = (int)(kv[ch] >> 24);
            }
#pragma unroll
            for (int ch = 0; ch < kWarpChunks; ++ch) {
                const unsigned V = __ballot_sync(FULL, vk[ch]);
                // same: lanes whose offset equals this lane's; m: lanes whose offset is this
                // lane's index
                unsigned same = V, m = V;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const unsigned bb = __ballot_sync(FULL, (dk[ch] >> b) & 1);
                    same &= ((dk[ch] >> b) & 1) ? bb : ~bb;
                    m &= bb ^ lb[b];
                }
                pos[ch] = __shfl_sync(FULL, bexcl, dk[ch]) + __shfl_sync(FULL, run, dk[ch]) +
                          __popc(same & lanemask_lt());
                run += __popc(m);
            }
            // parent slot of every kept entry: the last node whose first entry is at or
            // before it, by a branch-free binary search over nodeoff (L <= kWarpChunks * 32),
            // the chunks' searches interleaved so that their loads overlap
            int sl[kWarpChunks];
#pragma unroll
            for (int ch = 0; ch < kWarpChunks; ++ch) sl[ch] = 0;
            for (int st = L > 1 ? 1 << (31 - __clz(L - 1)) : 0; st > 0; st >>= 1) {
#pragma unroll
                for (int ch = 0; ch < kWarpChunks; ++ch) {
                    const int m = sl[ch] + st;
                    if (m < L && (int)FG_AT(R.nodeoff(wl), m, WN(uint16_t, WR_NODEOFF)) <=
                                     (int)(kv[ch] & 0xffffu))
                        sl[ch] = m;
                }
            }
#pragma unroll
            for (int ch = 0; ch < kWarpChunks; ++ch) {
                if (vk[ch]) {
                    FG_AT(R.sel(wl), pos[ch], WN(int32_t, WR_SEL)) =
                        (sl[ch] << 8) | (int)((kv[ch] >> 16) & 0xffu);
                    FG_AT(R.selped(wl), pos[ch], WN(int32_t, WR_SELPED)) = A + dk[ch];
                }
            }
            WPHASE(4);
        } else {
            // exact fallback: score the level again with exact PED offsets, find the K-th one
            // by bisection, compact the kept entries in enumeration order and rank them by
            // (PED, enumeration order)
            int dummy = 0;
            eval_level<Word, BK, FOLD, true>(p, R, L, n0, deg, n2, mrow, A, dummy);
            auto count_le = [&](int t) -> int {
                int cnt = 0;
                for (int k = lane; k < tot; k += 32)
                    cnt += ((int)FG_AT(R.ent(wl), k, WN(uint16_t, WR_ENT)) <= t);
                return warp_sum(cnt);
            };
            int lo = H - 1, hi = 0;
            for (int k = lane; k < tot; k += 32)
                hi = max(hi, (int)FG_AT(R.ent(wl), k, WN(uint16_t, WR_ENT)));
            hi = (int)__reduce_max_sync(FULL, (unsigned)hi);
            if (lo > hi) lo = hi;
            while (lo < hi) {   // count(<= lo - 1) < newL <= count(<= hi)
                const int mid = lo + (hi - lo) / 2;
                if (count_le(mid) >= newL) hi = mid;
                else lo = mid + 1;
            }
            const int T = lo;
            const int q = newL - (T > 0 ? count_le(T - 1) : 0);
            int keep_before = 0, eq_before = 0;
            for (int kb = 0; kb < tot; kb += 32) {
                const int k = kb + lane;
                const int d = k < tot ? (int)FG_AT(R.ent(wl), k, WN(uint16_t, WR_ENT)) : 0x10000;
                const bool is_eq = d == T;
                const unsigned eqb = __ballot_sync(FULL, is_eq);
                const bool keep = (d < T) || (is_eq && eq_before + __popc(eqb & lanemask_lt()) < q);
                const unsigned kbm = __ballot_sync(FULL, keep);
                if (keep)
                    FG_AT(R.klist(wl), keep_before + __popc(kbm & lanemask_lt()), WN(uint32_t, WR_KLIST)) =
                        ((uint32_t)d << 16) | (uint32_t)k;
                keep_before += __popc(kbm);
                eq_before += __popc(eqb);
            }
            __syncwarp();
            // rank of every kept key (keys are distinct: the entry index is in the low half)
            for (int x = lane; x < newL; x += 32) {
                const uint32_t kx = FG_AT(R.klist(wl), x, WN(uint32_t, WR_KLIST));
                int rank = 0;
                for (int y = 0; y < newL; ++y) rank += FG_AT(R.klist(wl), y, WN(uint32_t, WR_KLIST)) < kx;
                FG_AT(R.selped(wl), rank, WN(int32_t, WR_SELPED)) = (int)kx;
            }
            __syncwarp();
            for (int r = lane; r < newL; r += 32) {
                const uint32_t kx = (uint32_t)FG_AT(R.selped(wl), r, WN(int32_t, WR_SELPED));
                const int d = (int)(kx >> 16), k = (int)(kx & 0xffffu);
                const int s = node_of(p, R.nodeoff(wl), L, k);
                const int no = (int)FG_AT(R.nodeoff(wl), s, WN(uint16_t, WR_NODEOFF));
                const int t = k - no;
                const int cnt = (int)FG_AT(R.nodeoff(wl), s + 1, WN(uint16_t, WR_NODEOFF)) - no;
                int j = n2 + 1;      // record index: the deletion
                if (t < cnt - 1) {   // the t-th free target vertex of node s
                    const Word nmask = n2 >= WB ? ~(Word)0 : (((Word)1 << n2) - (Word)1);
                    Word x = ~FG_AT(R.imgc(wl), s, WN(Word, WR_IMG0)) & nmask;
                    for (int z = 0; z < t; ++z) x &= x - (Word)1;
                    j = ffs1(x);
                }
                FG_AT(R.sel(wl), r, WN(int32_t, WR_SEL)) = (s << 8) | j;
                FG_AT(R.selped(wl), r, WN(int32_t, WR_SELPED)) = A + d;
            }
            WPHASE(5);
        }
        __syncwarp();
        // kept children in key order (slot = rank): parent map + entry i, Img, PED, and the
        // g2 edges inside Img (for the leaf completion)
        {
            const int nvec = (i + 15) >> 4;
            const uint8_t *__restrict__ mapc = R.mapc(wl);
            uint8_t *__restrict__ mapn = R.mapn(wl);
            for (int r = lane; r < newL; r += 32) {
                const int v = FG_AT(R.sel(wl), r, WN(int32_t, WR_SEL));
                const int s = v >> 8, jr = v & 0xff, j = jr - 1;   // record index, vertex (n2: deletion)
                const int64_t src = (int64_t)s * (mrow >> 4), dst = (int64_t)r * (mrow >> 4);
                for (int t = 0; t < nvec; ++t)
                    FG_AT((uint4 *)mapn, dst + t, FG_N(uint4, wl.size[WR_MAP0])) =
                        FG_AT((const uint4 *)mapc, src + t, FG_N(uint4, wl.size[WR_MAP0]));
                FG_AT(mapn, (int64_t)r * mrow + i, wl.size[WR_MAP0]) = j < n2 ? (uint8_t)j : DEL;
                const Word im = FG_AT(R.imgc(wl), s, WN(Word, WR_IMG0));
                int e2 = FG_AT(R.e2c(wl), s, WN(uint16_t, WR_E20));
                Word imn = im;
                if (j < n2) {
                    e2 += popcw((Word)(FG_AT(R.tgt(wl), jr, WN(Rec, WR_TGT)).a2 & im));
                    imn |= (Word)1 << j;
                }
                FG_AT(R.imgn(wl), r, WN(Word, WR_IMG0)) = imn;
                FG_AT(R.e2n(wl), r, WN(uint16_t, WR_E20)) = (uint16_t)e2;
                FG_AT(R.pedn(wl), r, WN(int32_t, WR_PED0)) = FG_AT(R.selped(wl), r, WN(int32_t, WR_SELPED));
            }
        }
        __syncwarp();
        R.cur ^= 1;
        L = newL;
        WPHASE(6);
    }

    // ---- S5: complete every kept leaf (insert the free g2 vertices and their edges), least
    // (total, slot)
    unsigned long long best = ~0ull;
    for (int s = lane; s < L; s += 32) {
        const int nimg = popcw(FG_AT(R.imgc(wl), s, WN(Word, WR_IMG0)));
        const long long total = (long long)FG_AT(R.pedc(wl), s, WN(int32_t, WR_PED0)) +
                                (long long)c.vins * (n2 - nimg) +
                                (long long)c.eins * (m2.m - (int)FG_AT(R.e2c(wl), s, WN(uint16_t, WR_E20)));
        const unsigned long long key = ((unsigned long long)total << 32) | (unsigned)s;
        best = key < best ? key : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(FULL, best, o);
        best = y < best ? y : best;
    }
    if (lane == 0) {
        FG_AT(p.out_cost, pair, p.n_pairs) = (int32_t)(best >> 32);
        if (p.out_nevals) FG_AT(p.out_nevals, pair, p.n_pairs) = nevals + L;
    }
    const int bs = (int)(best & 0xffffffffull);
    const int64_t mo = FG_AT(p.map_off, pair, p.n_pairs);
    for (int k = lane; k < n1; k += 32) {
        const uint8_t v = FG_AT(R.mapc(wl), (int64_t)bs * mrow + k, wl.size[WR_MAP0]);
        FG_AT(p.out_map, mo + k, p.map_total) = v == DEL ? -1 : (int32_t)v;
    }
    __syncwarp();
    WPHASE(8);
#ifdef FASTGED_PHASE_TIMERS
    if (lane == 0 && p.phase_cycles)
        for (int k = 0; k < 16; ++k) atomicAdd(&p.phase_cycles[k], (unsigned long long)ph[k]);
#endif
#undef WN
}

// Persistent one-warp teams: each warp pops pairs from the class's queue until it is empty.
template <typename Word, int BK>
__global__ void __launch_bounds__(128, 5) kbest_warp_kernel(const KParams p)
{
    const int wic = (int)(threadIdx.x >> 5);
    const int gwarp = (int)blockIdx.x * (int)(blockDim.x >> 5) + wic;
    const uint32_t wb = (uint32_t)wic * (uint32_t)p.wl.warp_bytes;
    uint8_t *gw = p.wl.gmap ? p.gscratch + (int64_t)gwarp * p.wl.gmap_bytes : nullptr;
    const bool fold = p.cost.eins == p.cost.edel;
    for (;;) {
        int qi = 0;
        if ((threadIdx.x & 31) == 0) qi = atomicAdd(p.queue_head, 1);
        qi = __shfl_sync(0xffffffffu, qi, 0);
        if (qi >= p.n_order) break;
        const int pair = FG_AT(p.order, qi, p.n_order);
        if (fold) solve_pair_warp<Word, BK, true>(p, wb, gw, pair);
        else solve_pair_warp<Word, BK, false>(p, wb, gw, pair);
    }
}

template <typename Word, int BK>
static cudaError_t ensure_warp_attr()
{
    static bool done = false;
    if (done) return cudaSuccess;
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kbest_warp_kernel<Word, BK>);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kbest_warp_kernel<Word, BK>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) done = true;
    return e;
}

template <int BK>
cudaError_t launch_kbest_warp_bk(bool w32, const KParams &p, int grid, int block, size_t smem,
                                 cudaStream_t st)
{
    if (w32) {
        cudaError_t e = ensure_warp_attr<uint32_t, BK>();
        if (e != cudaSuccess) return e;
        kbest_warp_kernel<uint32_t, BK><<<grid, block, smem, st>>>(p);
    } else {
        cudaError_t e = ensure_warp_attr<uint64_t, BK>();
        if (e != cudaSuccess) return e;
        kbest_warp_kernel<uint64_t, BK><<<grid, block, smem, st>>>(p);
    }
    return cudaGetLastError();
}

template <int BK>
cudaError_t kbest_warp_occupancy_bk(bool w32, int block, size_t smem, int *out)
{
    if (w32) {
        cudaError_t e = ensure_warp_attr<uint32_t, BK>();
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, kbest_warp_kernel<uint32_t, BK>,
                                                             block, smem);
    }
    cudaError_t e = ensure_warp_attr<uint64_t, BK>();
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, kbest_warp_kernel<uint64_t, BK>,
                                                         block, smem);
}

}  // namespace fastged
