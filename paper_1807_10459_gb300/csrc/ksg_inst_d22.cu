// ksg_inst_d22.cu -- compiled specialisations of the fused KSG kernel for
// dx = 2, dy = 2, k = 4, 32 jobs per CTA, z buckets 1..6, 8, 10, 12, 16.
#include "ksg_list.cuh"

namespace idtx {

int ksg_variants_d22(KsgVariant *out)
{
    int n = 0;
    out[n++] = make_variant<2, 2, 1, 5, true, IDTX_FAST_QC, IDTX_FAST_NW>();
    out[n++] = make_variant<2, 2, 2, 5, true, IDTX_FAST_QC, IDTX_FAST_NW>();
    out[n++] = make_variant<2, 2, 3, 5, true, IDTX_FAST_QC, IDTX_FAST_NW>();
    out[n++] = make_variant<2, 2, 4, 5, true, IDTX_FAST_QC, IDTX_FAST_NW>();
    out[n++] = make_variant<2, 2, 5, 5, true, IDTX_FAST_QC, IDTX_FAST_NW>();
    out[n++] = make_variant<2, 2, 6, 5, true, IDTX_FAST_QC, IDTX_FAST_NW>();
    out[n++] = make_variant<2, 2, 8, 5, true, IDTX_FAST_QC, IDTX_FAST_NW>();
    out[n++] = make_variant<2, 2, 10, 5, true, IDTX_FAST_QC, IDTX_FAST_NW>();
    out[n++] = make_variant<2, 2, 12, 5, true, IDTX_FAST_QC, IDTX_FAST_NW>();
    out[n++] = make_variant<2, 2, 16, 5, true, IDTX_FAST_QC, IDTX_FAST_NW>();
    return n;
}

}  // namespace idtx
