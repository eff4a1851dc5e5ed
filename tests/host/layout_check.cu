// Host-side checks of the shared-memory layout helpers of the scan kernels
// (built and run by tests/test_layout_helpers.py; no GPU needed).
//   tslot / tstride: padded slots of the field-major scan trees
//   gstride:         spacing of the lane groups' shared-memory blocks
//   top_smem_bytes:  shared memory of the top-level scan's replay
//   ModelLayout:     the n <= 4 kernels' model area, read with vector loads
#include <cstdio>

#include "lqt_chain.cuh"
#include "lqt_kernels.cuh"
#include "lqt_variants.h"

using namespace lqt;
using lqt::chain::DownSmem;
using lqt::chain::FoldSmem;
using lqt::chain::RefoldSmem;
using lqt::chain::UpSmem;
using lqt::lanes::gstride;
using lqt::lanes::lds;

static int fails = 0;
#define CHECK(c, ...)                                   \
    do {                                                \
        if (!(c)) {                                     \
            std::printf("FAIL line %d: ", __LINE__);    \
            std::printf(__VA_ARGS__);                   \
            std::printf("\n");                          \
            ++fails;                                    \
        }                                               \
    } while (0)

// Largest number of distinct slots of one warp-wide access that share a bank:
// FP32 words over 32 banks per warp, FP64 words over 16 bank pairs per half-warp.
static int worst_bank_share(const int* slots, const bool* active, int es) {
    int worst = 1;
    const int phases = es == 8 ? 2 : 1, lanes = 32 / phases, banks = es == 8 ? 16 : 32;
    for (int ph = 0; ph < phases; ++ph)
        for (int b = 0; b < banks; ++b) {
            int distinct[32], nd = 0;
            for (int l = ph * lanes; l < (ph + 1) * lanes; ++l) {
                if (!active[l] || slots[l] % banks != b) continue;
                bool seen = false;
                for (int q = 0; q < nd; ++q) seen |= distinct[q] == slots[l];
                if (!seen) distinct[nd++] = slots[l];
            }
            if (nd > worst) worst = nd;
        }
    return worst;
}

// Every level of the left-anchored (slots 2ht, 2ht + h) and right-anchored
// (2ht + 2h - 1, 2ht + h - 1) sweeps of a W-slot tree, per warp.
template <typename R>
static void tree_checks(int W) {
    const int es = (int)sizeof(R), ts = tstride(W, es);
    int prev = -1;
    for (int i = 0; i < W; ++i) {
        const int s = tslot<R>(i);
        CHECK(s > prev && s < ts, "tslot es=%d W=%d i=%d -> %d (stride %d)", es, W, i, s, ts);
        prev = s;
    }
    CHECK((ts * es) % 16 == 0, "tree field of %d bytes is not a 16-byte multiple", ts * es);
    for (int h = 1; h < W; h <<= 1)
        for (int pat = 0; pat < 4; ++pat)
            for (int w0 = 0; w0 < W; w0 += 32) {
                int slots[32];
                bool active[32];
                for (int l = 0; l < 32; ++l) {
                    const int t = w0 + l;
                    const int base = pat < 2 ? t * 2 * h : t * 2 * h + 2 * h - 1;
                    const int i = base + ((pat == 1) ? h : (pat == 3) ? -h : 0);
                    const int top = pat < 2 ? t * 2 * h : t * 2 * h + 2 * h - 1;
                    active[l] = top < W && i >= 0 && i < W;
                    slots[l] = active[l] ? tslot<R>(i) : 0;
                }
                const int worst = worst_bank_share(slots, active, es);
                CHECK(worst == 1, "es=%d W=%d level h=%d pattern %d warp %d: %d-way conflict", es,
                      W, h, pat, w0 / 32, worst);
            }
}

// Column sweeps of the lane groups of a warp (lane r of group g reads element
// g * gstride + r * lds(N) + k): one bank per lane for FP32.
template <int N>
static void group_checks(int size) {
    const int st = gstride<N>(size);
    CHECK(st >= size && (st * 4) % 16 == 0, "gstride<%d>(%d) = %d", N, size, st);
    for (int k = 0; k < N; ++k) {
        int slots[32];
        bool active[32];
        for (int l = 0; l < 32; ++l) {
            const int g = l / N, r = l % N;
            slots[l] = g * st + r * lds(N) + k;
            active[l] = true;
        }
        const int worst = worst_bank_share(slots, active, 4);
        CHECK(worst == 1, "N=%d block %d: column %d has a %d-way conflict", N, size, k, worst);
    }
}


// The model area of the n <= 4 scan kernels: each part starts on a multiple of
// 4 elements and the parts do not overlap (p up to 2N), and the area starts
// 16 bytes into alignment in every kernel that places it (after the tree or
// staging area of k_bwd_up, k_bwd_down, k_fwd_down, k_solo), so that
// load_step's 16-byte vector loads of its parts are aligned.
template <typename R, int N, int M>
static void model_layout_checks() {
    using ML = ModelLayout<N, M>;
    constexpr int W = tile_threads<R, N, M>();
    using SM = Smem<R, N, M, W>;
    const int parts[] = {ML::OF, ML::OL, ML::OU, ML::OC, ML::OQ, ML::OHX};
    for (int o : parts) CHECK(o % 4 == 0, "N=%d M=%d: part at %d", N, M, o);
    CHECK(ML::OL >= ML::OF + N * N && ML::OU >= ML::OL + N * M && ML::OC >= ML::OU + M * M &&
              ML::OQ >= ML::OC + N && ML::OHX >= ML::OQ + Dims<N>::SYM,
          "N=%d M=%d: overlapping parts", N, M);
    for (int p = 0; p <= 2 * N; ++p) {
        CHECK(ML::OH(p) % 4 == 0 && ML::OH(p) >= ML::OHX + p * N, "N=%d p=%d: H part", N, p);
        CHECK(ML::size(p) % 4 == 0 && ML::size(p) >= ML::OH(p) + p * N, "N=%d p=%d: size", N, p);
    }
    const int bases[] = {SM::UP_BIG, SM::DOWN_BIG, SM::FDOWN_BIG, SoloSmem<R, N, M, W>::BIG};
    for (int b : bases) {
        const long long at = kSmemHead + (long long)(b + SM::RBUF) * (long long)sizeof(R);
        CHECK(at % 16 == 0, "N=%d M=%d W=%d: model area at byte %lld", N, M, W, at);
    }
}
#define MODEL_LAYOUT_CHECK(R, N, M) model_layout_checks<R, N, M>();

int main() {
    for (int W : {128, 256, 512}) tree_checks<float>(W);
    for (int W : {128, 256}) tree_checks<double>(W);  // FP64 tiles are at most 256 wide
    group_checks<4>(FoldSmem<4, 2, float>::SIZE);
    group_checks<4>(UpSmem<4>::SIZE);
    group_checks<8>(FoldSmem<8, 4, float>::SIZE);
    group_checks<8>(RefoldSmem<8, 4>::SIZE);
    group_checks<8>(UpSmem<8>::SIZE);
    group_checks<16>(FoldSmem<16, 8, float>::SIZE);
    group_checks<16>(RefoldSmem<16, 8>::SIZE);
    group_checks<16>(DownSmem<16>::SIZE);
    // the replayed top scan fits one CTA for every FP32 size (the headline path)
    CHECK(top_smem_bytes(Dims<1>::ELEM, Dims<1>::VALUE, 1, 256, 4, true) <= kTopSmemMax, "n=1");
    CHECK(top_smem_bytes(Dims<2>::ELEM, Dims<2>::VALUE, 2, 256, 4, true) <= kTopSmemMax, "n=2");
    CHECK(top_smem_bytes(Dims<3>::ELEM, Dims<3>::VALUE, 3, 256, 4, true) <= kTopSmemMax, "n=3");
    CHECK(top_smem_bytes(Dims<4>::ELEM, Dims<4>::VALUE, 4, 256, 4, true) <= kTopSmemMax, "n=4");
    LQT_VARIANTS_F32_SMALL(MODEL_LAYOUT_CHECK)
    LQT_VARIANTS_F32_N4(MODEL_LAYOUT_CHECK)
    LQT_VARIANTS_F64(MODEL_LAYOUT_CHECK)
    std::printf("%s (%d failures)\n", fails ? "layout checks FAILED" : "layout checks ok", fails);
    return fails ? 1 : 0;
}
