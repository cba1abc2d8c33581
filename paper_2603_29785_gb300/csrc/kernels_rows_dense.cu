// Compile-time row-kernel variants for the dense mode (stopband floor and
// remodulated tiles; Sec. III's undemodulated alternative): a tile spans the
// whole one-sided spectrum, so M >= N/2 + 1; M = 4320 = 2^5 3^3 5 is the
// smallest such length for 2 s segments at 4096 Hz (N = 8192).  Each entry
// also carries the ordinary (bisquare and window-table) kernels of its
// length.  Kept in their own translation unit so the library's objects
// compile in parallel; the registry in kernels_rows.cu lists them after its
// own variants.
#include "rows_common.cuh"

namespace qtam {
namespace {

#define QTAM_VD(M, NBS, MINB, ...) \
  make_variant_dense<StaticEngine<M, NBS, MINB, __VA_ARGS__>>(#M ":" #__VA_ARGS__ " rows/blk 2^" #NBS " minblk " #MINB)
const RowVariant kDenseVariants[] = {
    QTAM_VD(4320, 0, 3, 16, 18, 15),
    QTAM_VD(4320, 0, 4, 16, 18, 15),
    QTAM_VD(4320, 0, 2, 16, 27, 10),
};
#undef QTAM_VD

}  // namespace

int dense_row_variant_count() { return (int)(sizeof(kDenseVariants) / sizeof(kDenseVariants[0])); }
const RowVariant* dense_row_variant(int i) {
  return (i >= 0 && i < dense_row_variant_count()) ? &kDenseVariants[i] : nullptr;
}

}  // namespace qtam
