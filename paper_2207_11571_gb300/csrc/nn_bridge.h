// Interface between the solver and the forcing network (nn_*.cu).
#pragma once

#include "dg_common.h"

namespace dgnn {

// Runs the network on every element of state q (context c) and writes the forcing
// s[e][slot * n^3 + node] (float) for variables first_var .. first_var + n_vars - 1.
int nn_forcing_on_state(const nn_model* net, const dg_ctx* c, const double* q, float* s, int* first_var,
                        int* n_vars, cudaStream_t st, bool features_ready = false);

// Whether the network's input features of context c can be written by c's phase-A launch
// (the one-launch network path, every element in one tile batch, no padding columns); if
// so fills *out (the network's feature buffer, means and spreads).  The forcing is then
// evaluated with features_ready = true after that launch.
bool nn_phase_a_features(const nn_model* net, const dg_ctx* c, FeatureOut* out);

}  // namespace dgnn
