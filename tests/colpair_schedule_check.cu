// Host-side check of the index logic of the column-pair kernels
// (kzk_colpair.cuh) for every supported length ny = 2^L, 8 <= L <= 12:
//  * the radix schedule multiplies out to ny and ends at stride 1;
//  * freq (frequency at a position after the forward passes) and pos are
//    inverse permutations;
//  * in every pass the groups of all threads partition the elements, each
//    group being base + s j inside one block of R s elements, and a warp pass's
//    groups stay inside the warp's aligned 256 elements;
//  * the first pass's permuted rewrite (dense tile -> slots psw) only touches
//    8-element groups read by lanes of one warp;
//  * every shared-memory access of every pass is free of bank conflicts
//    (16-byte accesses: four phases of eight lanes, distinct 16-byte bank
//    groups within a phase), and so are the fused multiply's table reads
//    (pair_tab_row), up to one extra wavefront per warp at L = 8;
//  * pair_tab_row permutes the rows of a pair table within groups of 8 and
//    keeps the ny/2 + 1 folded rows inside pair_tab_rows(ny);
//  * the twiddle table of the schedule fits in ny entries.
// Prints "ok" and exits 0, else prints the first failure and exits 1.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../paper_2103_06080_b300/csrc/kzk_colpair.cuh"

using namespace kzk;

static int fails = 0;
#define CHECK(c, ...)                                   \
    do {                                                \
        if (!(c)) {                                     \
            if (fails++ < 10) {                         \
                std::printf("L=%d: ", L);               \
                std::printf(__VA_ARGS__);               \
                std::printf("\n");                      \
            }                                           \
        }                                               \
    } while (0)

// wavefronts of one 16-byte access by 32 lanes (slot < 0: lane idle)
static int wavefronts(const int* slot)
{
    int total = 0;
    for (int ph = 0; ph < 4; ph++) {
        int worst = 0;
        for (int g = 0; g < 8; g++) {
            int cnt = 0, seen[8], ns = 0;
            for (int l = 8 * ph; l < 8 * ph + 8; l++) {
                if (slot[l] < 0 || (slot[l] & 7) != g) continue;
                bool dup = false;
                for (int i = 0; i < ns; i++) dup |= seen[i] == slot[l];
                if (!dup) { seen[ns++] = slot[l]; cnt++; }
            }
            if (cnt > worst) worst = cnt;
        }
        total += worst;
    }
    return total;
}

template <int L, int I>
static void check_pass()
{
    using S = PairSched<L>;
    constexpr int N = S::N, T = S::T, R = S::radix(I), s = S::stride(I), G = 8 / R;
    std::vector<int> owner(N, -1);
    for (int t = 0; t < T; t++)
        for (int u = 0; u < G; u++) {
            int base, qq;
            pair_group<L, I>(t, u, base, qq);
            CHECK(qq >= 0 && qq < s, "pass %d: q %d out of [0, %d)", I, qq, s);
            CHECK(base % (R * s) == qq, "pass %d: base %d not at offset q of a block", I, base);
            for (int j = 0; j < R; j++) {
                const int e = base + s * j;
                CHECK(e >= 0 && e < N, "pass %d: element %d out of range", I, e);
                if (e < 0 || e >= N) continue;
                CHECK(owner[e] < 0, "pass %d: element %d in two groups", I, e);
                owner[e] = t;
                if (I >= S::NBP) CHECK(e / 256 == t / 32, "pass %d: warp pass leaves the warp's block", I);
            }
        }
    for (int e = 0; e < N; e++) CHECK(owner[e] >= 0, "pass %d: element %d in no group", I, e);
    if (I == 0)   // dense -> permuted rewrite: slot psw(e) holds element psw(e), read by the same warp
        for (int e = 0; e < N; e++)
            CHECK(owner[psw(e)] / 32 == owner[e] / 32, "first pass: slot of %d read by another warp", e);
    // bank conflicts: each (u, j) is one access instruction of every warp
    for (int w = 0; w < T / 32 || (w == 0 && T < 32); w++)
        for (int u = 0; u < G; u++)
            for (int j = 0; j < R; j++) {
                int slot[32];
                for (int l = 0; l < 32; l++) {
                    const int t = 32 * w + l;
                    if (t >= T) { slot[l] = -1; continue; }
                    int base, qq;
                    pair_group<L, I>(t, u, base, qq);
                    slot[l] = psw(base + s * j);
                }
                const int wf = wavefronts(slot);
                CHECK(wf <= 4, "pass %d: %d wavefronts for one access (u %d, j %d, warp %d)", I, wf, u, j, w);
            }
}

template <int L>
static void check_length()
{
    using S = PairSched<L>;
    constexpr int N = S::N;
    int prod = 1;
    for (int i = 0; i < S::NP; i++) prod *= S::radix(i);
    CHECK(prod == N, "radices multiply to %d", prod);
    CHECK(S::stride(S::NP - 1) == 1, "last stride %d", S::stride(S::NP - 1));
    CHECK(S::stride(S::NBP) == 32 && S::radix(S::NBP) == 8, "first warp pass");
    CHECK(S::TW <= N, "twiddle table %d > %d", S::TW, N);
    std::vector<int> hit(N, 0);
    for (int p = 0; p < N; p++) {
        const int k = S::freq(p);
        CHECK(k >= 0 && k < N, "freq(%d) = %d", p, k);
        if (k >= 0 && k < N) hit[k]++;
        CHECK(S::pos(k) == p, "pos(freq(%d)) = %d", p, S::pos(k));
    }
    for (int k = 0; k < N; k++) CHECK(hit[k] == 1, "frequency %d hit %d times", k, hit[k]);
    // pair-table rows
    const int rows = pair_tab_rows(N);
    std::vector<int> tr(rows, 0);
    for (int r = 0; r < rows; r++) {
        const int x = pair_tab_row<L>(r);
        CHECK(x >= 0 && x < rows && (x >> 3) == (r >> 3), "pair_tab_row(%d) = %d", r, x);
        if (x >= 0 && x < rows) tr[x]++;
    }
    for (int x = 0; x < rows; x++) CHECK(tr[x] == 1, "table row %d hit %d times", x, tr[x]);
    // fused multiply's table reads: lane l of warp w reads the rows of positions 256 w + 8 l + j
    int extra = 0;
    for (int w = 0; w < N / 256; w++)
        for (int j = 0; j < 8; j++) {
            int slot[32];
            for (int l = 0; l < 32; l++) {
                const int k = S::freq(256 * w + 8 * l + j);
                slot[l] = pair_tab_row<L>(k <= N / 2 ? k : N - k);
            }
            extra += wavefronts(slot) - 4;
        }
    CHECK(extra <= (L == 8 ? 1 : 0), "table reads: %d extra wavefronts", extra);
    check_pass<L, 0>();
    check_pass<L, 1>();
    check_pass<L, 2>();
    if constexpr (S::NP > 3) check_pass<L, 3>();
    if constexpr (S::NP > 4) check_pass<L, 4>();
}

int main()
{
    check_length<8>();
    check_length<9>();
    check_length<10>();
    check_length<11>();
    check_length<12>();
    if (fails) {
        std::printf("%d failures\n", fails);
        return 1;
    }
    std::printf("ok\n");
    return 0;
}
