// Compile-time row-kernel variants added after measuring the first registry
// against the workloads:
// - balanced radix sequences for the short envelope lengths of the uneven
//   batch (M = 75 ... 1200, segments of 1-16 s), whose stages hold about the
//   same number of butterfly items, so few threads of a block sit idle in
//   any stage;
// - a four-stage sequence at M = 8192 (16·8·8·8) that fits in 64 registers,
//   so two 512-thread blocks share an SM where the three-stage sequences
//   (96-99 registers) allowed one;
// - at M = 2400, 16·10·15 on 160 threads (the 10-point stage in two rounds)
//   in place of 256, at 6 blocks per SM.
// Kept in their own translation unit so the library's objects compile in
// parallel; the registry in kernels_rows.cu lists them after the row-pair
// variants.
#include "rows_common.cuh"

namespace qtam {
namespace {

// Measured per length against the older shapes (forward + inverse of one
// launch over 38-48 segments at 4096 Hz, Q {8,16,32} x 128 rows): M = 1200
// 0.142 against 0.200 ms, M = 600 0.081 against 0.121 ms (2 rows per
// 64-thread block; 0.087 at 4 rows per block), M = 300 0.054 against 0.066
// ms (2 rows per block, 12 blocks per SM), M = 150 0.049 against 0.053 ms;
// at M = 75 the two shapes trade places with the sample rate, so the older
// one stays the default.  Fewer rows per block with more blocks per SM won
// at every short length: a block's barrier then waits on fewer threads.  At
// M = 8192 (64 s segments, Q {4..64} x 128 rows, 64 segments, FP32
// envelopes) 16·8·8·8 at 2 blocks per SM takes 1.010 + 0.889 ms against
// 1.215 + 1.315 ms for 16·16·32 at one block.  At M = 2400 (32 s segments,
// Q {8,16,32} x 128 rows) the 160-thread block takes 0.107 + 0.105 ms for 43
// segments at 4096 Hz against 0.119 + 0.124 ms for the 256-thread one, and
// 0.132 + 0.144 against 0.144 + 0.168 ms for 55 segments at 16384 Hz.  The
// 4800-point kernel on 160 threads (two rounds in every stage, 114-117
// registers) lost: 0.560 + 0.857 against 0.509 + 0.487 ms.  The first
// preferred entry of a length is its default for bisquare plans; the tuner
// times all of them.
template <class Eng> RowVariant make_variant_pref(const char* name) {
  RowVariant v = make_variant<Eng>(name);
  v.preferred = 1;
  return v;
}
#define QTAM_VS_NT(NT, M, NBS, MINB, ...)                                                                        \
  make_variant_pref<ThreadsEngine<NT, M, NBS, MINB, __VA_ARGS__>>(#M ":" #__VA_ARGS__ " rows/blk 2^" #NBS " minblk " \
                                                                  #MINB " threads " #NT)
#define QTAM_VS(M, NBS, MINB, ...) \
  make_variant_pref<StaticEngine<M, NBS, MINB, __VA_ARGS__>>(#M ":" #__VA_ARGS__ " rows/blk 2^" #NBS " minblk " #MINB)
#define QTAM_VN(M, NBS, MINB, ...) \
  make_variant<StaticEngine<M, NBS, MINB, __VA_ARGS__>>(#M ":" #__VA_ARGS__ " rows/blk 2^" #NBS " minblk " #MINB)
const RowVariant kTunedVariants[] = {
    QTAM_VS(1200, 0, 8, 10, 12, 10),
    QTAM_VS(1200, 0, 6, 10, 12, 10),
    QTAM_VS(600, 1, 8, 25, 24),
    QTAM_VS(600, 2, 4, 25, 24),
    QTAM_VS(600, 2, 3, 24, 25),
    QTAM_VS(300, 1, 12, 15, 20),
    QTAM_VS(300, 2, 4, 15, 20),
    QTAM_VS(300, 3, 2, 15, 20),
    QTAM_VS(150, 3, 4, 10, 15),
    QTAM_VS(150, 4, 2, 10, 15),
    QTAM_VN(75, 4, 3, 5, 15),
    QTAM_VS(8192, 0, 2, 16, 8, 8, 8),
    QTAM_VN(8192, 0, 2, 16, 16, 8, 4),
    QTAM_VS_NT(160, 2400, 0, 6, 16, 10, 15),
};
#undef QTAM_VN
#undef QTAM_VS_NT
#undef QTAM_VS

}  // namespace

int tuned_row_variant_count() { return (int)(sizeof(kTunedVariants) / sizeof(kTunedVariants[0])); }
const RowVariant* tuned_row_variant(int i) {
  return (i >= 0 && i < tuned_row_variant_count()) ? &kTunedVariants[i] : nullptr;
}

}  // namespace qtam
