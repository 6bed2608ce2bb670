// HSS entry points (filled in by the compression / ULV sources).
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
    o->reserved = 0;
}

int hss_compress(krr_ctx *, const float *, int64_t, int32_t, const krr_options *, krr_hss **out) {
    if (out) *out = nullptr;
    return fail(KRR_ERR_NOT_IMPLEMENTED, "hss_compress");
}
int hss_update_lambda(krr_hss *, double) { return fail(KRR_ERR_NOT_IMPLEMENTED, "hss_update_lambda"); }
int hss_factor(krr_hss *) { return fail(KRR_ERR_NOT_IMPLEMENTED, "hss_factor"); }
int hss_solve(krr_hss *, const double *, int32_t, int64_t, double *, int64_t, double, int32_t, double *) {
    return fail(KRR_ERR_NOT_IMPLEMENTED, "hss_solve");
}
int krr_predict(krr_hss *, const float *, int64_t, const double *, int32_t, int64_t, double *, int64_t) {
    return fail(KRR_ERR_NOT_IMPLEMENTED, "krr_predict");
}
int hss_stats(const krr_hss *, krr_hss_stats *) { return fail(KRR_ERR_NOT_IMPLEMENTED, "hss_stats"); }
const int32_t *hss_permutation(const krr_hss *) { return nullptr; }
void hss_destroy(krr_hss *) {}

}  // extern "C"
