// ion_ext.cu -- per-flag extensions of a simulation handle (persistent, surrogate) and
// the batched / training entry points.
#include <cuda_runtime.h>

#include "ion.h"
#include "ion_sim.h"

ion_status ion_sim_setup_extras(ion_sim *s, const ion_params *p) {
    (void)p;
    if (s->flags & ION_FLAG_SURROGATE) return ion_fail(nullptr, ION_ERR_UNSUPPORTED, "surrogate: not built");
    return ION_OK;
}

extern "C" ion_status ion_create_batch(int32_t n_nets, const ion_net *nets, const ion_conn *conns,
                                       const ion_params *params, const float *init_state, ion_sim **out) {
    (void)n_nets; (void)nets; (void)conns; (void)params; (void)init_state;
    if (out) *out = nullptr;
    return ion_fail(nullptr, ION_ERR_UNSUPPORTED, "ion_create_batch: not built");
}

extern "C" ion_status ion_surrogate_train(const ion_train_cfg *cfg, ion_surrogate_weights *w, float *loss) {
    (void)cfg; (void)w; (void)loss;
    return ion_fail(nullptr, ION_ERR_UNSUPPORTED, "ion_surrogate_train: not built");
}
