// ksg_inst_generic.cu -- the catch-all specialisation of the fused KSG kernel:
// any k <= 15 (runtime), dx <= 4, dy <= 4, dz <= 16 (zero-padded), 32 jobs x 16 queries per CTA, 8 warps.
#include "ksg_list.cuh"

namespace idtx {

int ksg_variants_generic(KsgVariant *out)
{
    int n = 0;
    out[n++] = make_variant<4, 4, 16, 16, false, 16, 8>();
    return n;
}

}  // namespace idtx
