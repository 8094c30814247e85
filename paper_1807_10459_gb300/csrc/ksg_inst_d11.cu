// ksg_inst_d11.cu -- compiled specialisations of the fused KSG kernel for
// dx = 1, dy = 1, k = 4, 32 jobs per CTA, z buckets 1..6, 8, 10, 12, 16.
#include "ksg_list.cuh"

namespace idtx {

int ksg_variants_d11(KsgVariant *out)
{
    int n = 0;
    out[n++] = make_variant<1, 1, 1, 5, true, IDTX_FAST_QC, IDTX_FAST_NW>();
    out[n++] = make_variant<1, 1, 2, 5, true, IDTX_FAST_QC, IDTX_FAST_NW>();
    out[n++] = make_variant<1, 1, 3, 5, true, IDTX_FAST_QC, IDTX_FAST_NW>();
    out[n++] = make_variant<1, 1, 4, 5, true, IDTX_FAST_QC, IDTX_FAST_NW>();
    out[n++] = make_variant<1, 1, 5, 5, true, IDTX_FAST_QC, IDTX_FAST_NW>();
    out[n++] = make_variant<1, 1, 6, 5, true, IDTX_FAST_QC, IDTX_FAST_NW>();
    out[n++] = make_variant<1, 1, 8, 5, true, IDTX_FAST_QC, IDTX_FAST_NW>();
    out[n++] = make_variant<1, 1, 10, 5, true, IDTX_FAST_QC, IDTX_FAST_NW>();
    out[n++] = make_variant<1, 1, 12, 5, true, IDTX_FAST_QC, IDTX_FAST_NW>();
    out[n++] = make_variant<1, 1, 16, 5, true, IDTX_FAST_QC, IDTX_FAST_NW>();
    return n;
}

}  // namespace idtx
