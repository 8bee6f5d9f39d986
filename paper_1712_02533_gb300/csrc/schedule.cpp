// Scan schedules (host).  Each schedule turns N slots holding x_0..x_{N-1}
// into inclusive prefixes data[e] = x_0 (.) ... (.) x_e for an operator that is
// only approximately associative, so the op list fixes the bracketing.  Ops of
// one level read the values held before the level (level-synchronous, i.e. the
// double buffering the paper prescribes for Kogge-Stone).  Slots >= N are
// auxiliary.  Algorithms from Chapter "Prefix sum" (serial, Blelloch,
// Brent-Kung, Kogge-Stone, Sklansky, and the Han-Carlson hybrid of Section
// "Other work") and Chapter "Distributed prefix sum" (general strategy,
// inclusive global scan, alternative strategy).
#include "schedule.h"

#include <algorithm>

namespace regsched {

static int clog2(int n)
{
    int k = 0;
    while ((1 << k) < n) k++;
    return k;
}

static void add(Schedule &s, int lv, int kind, int dst, int a, int b)
{
    if ((int)s.levels.size() <= lv) s.levels.resize(lv + 1);
    s.levels[lv].push_back(Op{kind, dst, a, b});
}

// data[i] = data[i-1] (.) data[i]
static void serial(Schedule &s, int n, int base)
{
    int lv = (int)s.levels.size();
    for (int i = 1; i < n; i++) add(s, lv++, OP_COMBINE, base + i, base + i - 1, base + i);
}

// step i: every j >= 2^i combines with j - 2^i
static void kogge_stone(Schedule &s, int n, int base)
{
    int lv = (int)s.levels.size();
    for (int i = 0; i < clog2(n); i++, lv++) {
        int st = 1 << i;
        for (int j = st; j < n; j++) add(s, lv, OP_COMBINE, base + j, base + j - st, base + j);
    }
}

// step i: source j = 2^i - 1 + m 2^{i+1} feeds the following 2^i slots
static void sklansky(Schedule &s, int n, int base)
{
    int lv = (int)s.levels.size();
    for (int i = 0; i < clog2(n); i++, lv++) {
        int st = 1 << i;
        s.levels.resize(lv + 1);
        for (int j = st - 1; j < n; j += 2 * st)
            for (int k = 0; k < st; k++)
                if (j + k + 1 < n) add(s, lv, OP_COMBINE, base + j + k + 1, base + j, base + j + k + 1);
    }
}

// tree up-sweep: data[j] = data[j - 2^i] (.) data[j], j = 2^{i+1}-1 step 2^{i+1}
static void upsweep(Schedule &s, int n, const std::vector<int> &slot)
{
    for (int i = 0; i < clog2(n); i++) {
        int st = 1 << i;
        bool any = false;
        int lv = (int)s.levels.size();
        for (int j = 2 * st - 1; j < n; j += 2 * st) {
            add(s, lv, OP_COMBINE, slot[j], slot[j - st], slot[j]);
            any = true;
        }
        (void)any;
    }
}

static void brent_kung(Schedule &s, int n, int base)
{
    std::vector<int> slot(n);
    for (int e = 0; e < n; e++) slot[e] = base + e;
    upsweep(s, n, slot);
    // breadth-first down-sweep: data[j + 2^i - 1] = data[j - 1] (.) data[j + 2^i - 1]
    for (int i = clog2(n) - 2; i >= 0; i--) {
        int st = 1 << i;
        int lv = (int)s.levels.size();
        bool any = false;
        for (int j = 2 * st; j + st - 1 < n; j += 2 * st) {
            add(s, lv, OP_COMBINE, base + j + st - 1, base + j - 1, base + j + st - 1);
            any = true;
        }
        (void)any;
    }
}

// Blelloch exclusive scan over n elements padded to a power of two P with
// identity slots aux .. aux+P-n-1; slot aux+P-n saves the root's reduction.
// Down-sweep: left child <- parent; right child <- parent (.) old left child
// (the prefix stays on the left, as a non-commutative operator needs).
static void blelloch_excl(Schedule &s, int n, int base, int aux, std::vector<int> &slot, int &total)
{
    int P = 1 << clog2(n);
    slot.resize(P);
    for (int e = 0; e < P; e++) slot[e] = e < n ? base + e : aux + (e - n);
    total = aux + (P - n);
    if (P > n) {
        int lv = (int)s.levels.size();
        for (int e = n; e < P; e++) add(s, lv, OP_IDENTITY, slot[e], -1, -1);
    }
    for (int i = 0; i < clog2(P); i++) {
        int st = 1 << i;
        int lv = (int)s.levels.size();
        for (int j = 2 * st - 1; j < P; j += 2 * st) add(s, lv, OP_COMBINE, slot[j], slot[j - st], slot[j]);
    }
    int lv = (int)s.levels.size();
    add(s, lv, OP_COPY, total, slot[P - 1], -1);
    add(s, lv, OP_IDENTITY, slot[P - 1], -1, -1);
    for (int i = clog2(P) - 1; i >= 0; i--) {
        int st = 1 << i;
        lv = (int)s.levels.size();
        for (int j = 0; j < P; j += 2 * st) {
            int left = slot[j + st - 1], right = slot[j + 2 * st - 1];
            add(s, lv, OP_COPY, left, right, -1);
            add(s, lv, OP_COMBINE, right, right, left);
        }
    }
}

static void blelloch(Schedule &s, int n, int base)
{
    std::vector<int> slot;
    int total;
    blelloch_excl(s, n, base, base + n, slot, total);
    int lv = (int)s.levels.size();
    for (int e = 0; e + 1 < n; e++) add(s, lv, OP_COPY, base + e, slot[e + 1], -1);
    add(s, lv, OP_COPY, base + n - 1, total, -1);
}

// Han-Carlson hybrid (Section "Other work": Brent-Kung and Kogge-Stone merged,
// parameter k, span log2 N + k): the first k up-sweep levels of the tree reduce
// blocks of 2^k elements; Kogge-Stone runs over the last elements of the
// complete blocks, which then hold their prefixes; the last k down-sweep levels
// of the tree fill in the rest (the elements of an incomplete last block too).
// k = 1 is the classic adder; k >= log2 N gives Brent-Kung.
//
// Ladner-Fischer(k) (the same section: Sklansky and Brent-Kung combined) is the
// same construction with Sklansky's tree over the block ends instead of
// Kogge-Stone: span log2 N + k at less work than Sklansky; k = 0 is Sklansky.
static void block_hybrid(Schedule &s, int n, int k, int base, bool sklansky_middle)
{
    k = std::max(sklansky_middle ? 0 : 1, std::min(k, clog2(n)));
    for (int i = 0; i < k; i++) {
        const int st = 1 << i, lv = (int)s.levels.size();
        for (int j = 2 * st - 1; j < n; j += 2 * st) add(s, lv, OP_COMBINE, base + j, base + j - st, base + j);
    }
    const int blk = 1 << k, m = n / blk;  // block t (t < m) ends at (t + 1) blk - 1
    auto end = [&](int t) { return base + (t + 1) * blk - 1; };
    for (int i = 0; i < clog2(m); i++) {
        const int st = 1 << i, lv = (int)s.levels.size();
        if (sklansky_middle) {
            // block end src = st - 1 + q 2 st feeds the following st block ends
            for (int src = st - 1; src < m; src += 2 * st)
                for (int t = src + 1; t <= src + st && t < m; t++) add(s, lv, OP_COMBINE, end(t), end(src), end(t));
        } else {
            for (int t = st; t < m; t++) add(s, lv, OP_COMBINE, end(t), end(t - st), end(t));
        }
    }
    for (int i = k - 1; i >= 0; i--) {
        const int st = 1 << i, lv = (int)s.levels.size();
        for (int j = 2 * st; j + st - 1 < n; j += 2 * st) add(s, lv, OP_COMBINE, base + j + st - 1, base + j - 1, base + j + st - 1);
    }
}

static int pow2ceil(int n) { return 1 << clog2(n); }

int aux_slots(int kind, int n, int chunks, int global_kind)
{
    if (kind == K_BLELLOCH) return pow2ceil(n) - n + 1;
    if (kind == K_CHUNKED || kind == K_CHUNKED_ALT) {
        int p = std::max(1, std::min(chunks, n));
        int extra = global_kind == K_BLELLOCH ? pow2ceil(p) - p + 1 : 0;
        return p + extra;
    }
    return 0;
}

static void global_scan(Schedule &s, int kind, int p, int gbase)
{
    switch (kind) {
    case K_SERIAL: serial(s, p, gbase); break;
    case K_SKLANSKY: sklansky(s, p, gbase); break;
    case K_KOGGE_STONE: kogge_stone(s, p, gbase); break;
    case K_BRENT_KUNG: brent_kung(s, p, gbase); break;
    default: break;
    }
}

// chunk I gets floor(N/P)+1 elements for I < N mod P, else floor(N/P)
static std::vector<std::pair<int, int>> chunk_bounds(int n, int p)
{
    std::vector<std::pair<int, int>> b;
    int k = n / p, rem = n % p, l = 0;
    for (int i = 0; i < p; i++) {
        int sz = k + (i < rem ? 1 : 0);
        b.push_back({l, l + sz - 1});
        l += sz;
    }
    return b;
}

// General strategy: local serial scans, global scan of chunk totals, then
// every element of chunk I >= 1 combined with the exclusive global value; an
// inclusive global algorithm hands the inclusive value to the chunk's last
// element directly.
static void chunked(Schedule &s, int n, int chunks, int gkind, int base)
{
    int p = std::max(1, std::min(chunks, n));
    auto bnd = chunk_bounds(n, p);
    int gbase = base + n, gaux = gbase + p;
    int kmax = 0;
    for (auto &c : bnd) kmax = std::max(kmax, c.second - c.first + 1);
    for (int t = 1; t < kmax; t++) {
        int lv = (int)s.levels.size();
        for (auto &c : bnd)
            if (c.first + t <= c.second) add(s, lv, OP_COMBINE, base + c.first + t, base + c.first + t - 1, base + c.first + t);
    }
    if (p == 1) return;
    int lv = (int)s.levels.size();
    for (int i = 0; i < p; i++) add(s, lv, OP_COPY, gbase + i, base + bnd[i].second, -1);
    std::vector<Op> stage2;
    if (gkind == K_BLELLOCH) {
        std::vector<int> gslot;
        int total;
        blelloch_excl(s, p, gbase, gaux, gslot, total);
        for (int i = 1; i < p; i++)
            for (int e = bnd[i].first; e <= bnd[i].second; e++) stage2.push_back(Op{OP_COMBINE, base + e, gslot[i], base + e});
    } else {
        global_scan(s, gkind, p, gbase);
        for (int i = 1; i < p; i++) {
            for (int e = bnd[i].first; e < bnd[i].second; e++) stage2.push_back(Op{OP_COMBINE, base + e, gbase + i - 1, base + e});
            stage2.push_back(Op{OP_COPY, base + bnd[i].second, gbase + i, -1});
        }
    }
    s.levels.push_back(stage2);
}

// Alternative strategy (reduce-then-scan): chunk totals by reduction, an
// exclusive scan of the totals, then per chunk: first element combined with
// the exclusive value and a serial rescan.
static void chunked_alt(Schedule &s, int n, int chunks, int gkind, int base)
{
    int p = std::max(1, std::min(chunks, n));
    if (p == 1) {
        serial(s, n, base);
        return;
    }
    auto bnd = chunk_bounds(n, p);
    int gbase = base + n, gaux = gbase + p;
    int lv = (int)s.levels.size();
    for (int i = 0; i < p; i++) add(s, lv, OP_COPY, gbase + i, base + bnd[i].first, -1);
    int kmax = 0;
    for (auto &c : bnd) kmax = std::max(kmax, c.second - c.first + 1);
    for (int t = 1; t < kmax; t++) {
        lv = (int)s.levels.size();
        for (int i = 0; i < p; i++)
            if (bnd[i].first + t <= bnd[i].second) add(s, lv, OP_COMBINE, gbase + i, gbase + i, base + bnd[i].first + t);
    }
    std::vector<int> excl(p, -1);
    if (gkind == K_BLELLOCH) {
        std::vector<int> gslot;
        int total;
        blelloch_excl(s, p, gbase, gaux, gslot, total);
        for (int i = 0; i < p; i++) excl[i] = gslot[i];
    } else {
        global_scan(s, gkind, p, gbase);
        for (int i = 1; i < p; i++) excl[i] = gbase + i - 1;
    }
    lv = (int)s.levels.size();
    for (int i = 1; i < p; i++) add(s, lv, OP_COMBINE, base + bnd[i].first, excl[i], base + bnd[i].first);
    for (int t = 1; t < kmax; t++) {
        lv = (int)s.levels.size();
        for (auto &c : bnd)
            if (c.first + t <= c.second) add(s, lv, OP_COMBINE, base + c.first + t, base + c.first + t - 1, base + c.first + t);
    }
}

bool make_schedule(int kind, int n, int chunks, int global_kind, Schedule &out)
{
    out.levels.clear();
    if (n <= 1) return true;
    switch (kind) {
    case K_SERIAL: serial(out, n, 0); break;
    case K_SKLANSKY: sklansky(out, n, 0); break;
    case K_KOGGE_STONE: kogge_stone(out, n, 0); break;
    case K_BRENT_KUNG: brent_kung(out, n, 0); break;
    case K_BLELLOCH: blelloch(out, n, 0); break;
    case K_HAN_CARLSON: block_hybrid(out, n, chunks, 0, false); break;
    case K_LADNER_FISCHER: block_hybrid(out, n, chunks, 0, true); break;
    case K_CHUNKED:
        if (global_kind < 0 || global_kind > K_BLELLOCH) return false;
        chunked(out, n, chunks, global_kind, 0);
        break;
    case K_CHUNKED_ALT:
        if (global_kind < 0 || global_kind > K_BLELLOCH) return false;
        chunked_alt(out, n, chunks, global_kind, 0);
        break;
    default: return false;
    }
    // drop empty levels
    std::vector<std::vector<Op>> lv;
    for (auto &l : out.levels)
        if (!l.empty()) lv.push_back(l);
    out.levels.swap(lv);
    return true;
}

}  // namespace regsched
