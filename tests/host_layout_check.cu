// Host-side checks of the layout arithmetic the kernels share (no kernel is
// launched; runs on any machine): the map between the network's exchange
// output layout (K lobes) and the kernels' internal layout of KM = 8 or 16
// lobes, the disabled-lobe rows, the core-matrix tile offsets of the
// tensor-core operands, and the shared-memory and TMEM budgets of the
// kernels.  Prints "ok" and exits 0 when every check holds.
#include <cstdio>
#include <set>

#include "../paper_2410_18944_gb300/csrc/field.cuh"
#include "../paper_2410_18944_gb300/csrc/umma.cuh"

using namespace wost;

static int failures = 0;
#define CHECK(cond)                                                             \
    do {                                                                        \
        if (!(cond)) {                                                          \
            if (failures < 20) std::printf("failed: %s (line %d)\n", #cond, __LINE__); \
            ++failures;                                                         \
        }                                                                       \
    } while (0)

static void check_output_layout(int KM) {
    for (int d = 2; d <= 3; ++d) {
        CHECK((d + 2) * KM + 1 <= out_pad(KM));
        CHECK(out_pad(KM) % 16 == 0);
        for (int K = 1; K <= KM; ++K) {
            const int nout = (d + 2) * K + 1;
            std::set<int> rows;
            for (int e = 0; e < nout; ++e) {
                const int r = exchange_to_out_row(e, d, K, KM);
                CHECK(r >= 0 && r < out_pad(KM));
                CHECK(out_row_to_exchange(r, d, K, KM) == e);
                rows.insert(r);
            }
            CHECK((int)rows.size() == nout);
            int mapped = 0, off = 0;
            for (int r = 0; r < out_pad(KM); ++r) {
                const int e = out_row_to_exchange(r, d, K, KM);
                if (e >= 0) {
                    ++mapped;
                    CHECK(exchange_to_out_row(e, d, K, KM) == r);
                }
                if (is_off_lambda(r, d, K, KM)) {
                    ++off;
                    CHECK(e < 0);
                    // a lambda' row of a lobe past K
                    CHECK(r >= KM * d + KM + K && r < KM * d + 2 * KM);
                }
            }
            CHECK(mapped == nout);
            CHECK(off == KM - K);
            // the selection logit sits right after the lambda' rows
            CHECK(exchange_to_out_row(nout - 1, d, K, KM) == KM * (d + 2));
        }
    }
    CHECK(field_km(1) == kMaxK && field_km(kMaxK) == kMaxK && field_km(kMaxK + 1) == kMaxKWide &&
          field_km(kMaxKWide) == kMaxKWide);
}

static void check_core_matrix_offsets() {
    const int widths[] = {32, 48, 64, 96, 128, 160};
    for (int C : widths) {
        std::set<unsigned> seen;
        for (int r = 0; r < 128; ++r)
            for (int c = 0; c < C; ++c) {
                const unsigned o = cm_offset(r, c, C);
                CHECK(o % 2 == 0 && o < 128u * C * 2u);
                seen.insert(o);
                // 8 consecutive columns of a row are one 16-byte vector
                if (c % 8 == 0) CHECK(o % 16 == 0 && cm_offset(r, c + 7, C) == o + 14);
            }
        CHECK((int)seen.size() == 128 * C);
    }
}

static void check_budgets() {
    for (unsigned n : {1u, 32u, 33u, 64u, 96u, 128u, 200u, 256u, 320u, 512u}) {
        const unsigned c = tmem_cols(n);
        CHECK(c >= n && c >= 32 && (c & (c - 1)) == 0 && c <= 512);
    }
    CHECK(tile_tmem_cols(kMaxK) >= out_pad(kMaxK) && tile_tmem_cols(kMaxKWide) >= out_pad(kMaxKWide));
    CHECK(2 * tile_tmem_cols(kMaxKWide) <= 512);
    CHECK(wimg_bytes(kMaxK) % 16 == 0 && wimg_bytes(kMaxKWide) % 16 == 0);
    CHECK(cta_tiles_smem(kMaxKWide) <= 227 * 1024);
}

int main() {
    check_output_layout(kMaxK);
    check_output_layout(kMaxKWide);
    check_core_matrix_offsets();
    check_budgets();
    if (failures) {
        std::printf("%d checks failed\n", failures);
        return 1;
    }
    std::printf("ok\n");
    return 0;
}
