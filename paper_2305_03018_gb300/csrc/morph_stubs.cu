// Entry points declared in morph.h whose implementation is not in this build yet.
#include "morph_internal.h"

extern "C" {
int morph_run_batch(morph_ctx*, const morph_problem*, int, const morph_opts*, morph_stream_t) {
    return MORPH_E_UNSUPPORTED;
}
int morph_batch_capture(morph_ctx*, const morph_problem*, int, const morph_opts*, morph_batch** out) {
    if (out) *out = nullptr;
    return MORPH_E_UNSUPPORTED;
}
int morph_batch_launch(morph_batch*, morph_stream_t) { return MORPH_E_UNSUPPORTED; }
int morph_batch_destroy(morph_batch*) { return MORPH_E_UNSUPPORTED; }
}
