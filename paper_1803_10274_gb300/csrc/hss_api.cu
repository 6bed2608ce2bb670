// Default options of the HSS path.
#include "common.cuh"

using namespace krr;

extern "C" {

void krr_default_options(krr_options *o) {
    if (!o) return;
    o->h = 1.0;
    o->lambda = 1.0;
    o->eps_c = 0.03;
    o->eps_abs = 0.0;
    o->leaf = 128;
    o->r0 = 64;
    o->p = 10;
    o->r_max = 2048;
    o->seed = 1;
    o->precision = KRR_MIXED;
    o->flags = 0;
    o->ordering = KRR_ORDER_TWO_MEANS;
    o->pad = 0;
}

}  // extern "C"
