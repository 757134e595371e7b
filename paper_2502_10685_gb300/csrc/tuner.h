// tuner.h -- the path tuner's hooks into context creation (not part of the
// public interface).
#pragma once

#include "../../include/stab.h"

namespace stab {

// The choice an AUTO context of n qubits on `device` runs with: the cached
// entry for the GPU's name, else (STAB_PATH_TUNE not 0) measured now and
// cached, else the defaults.  `like` (may be NULL) gives the probe contexts
// the creating context's allocator hooks (they run on streams of their own).
int resolve_path_choice(int device, int n, const stab_opts *like, stab_path_choice *out);

// Creates a context that runs with `choice` instead of consulting the cache
// (the tuner's candidates).
int create_with_choice(int n, const stab_opts *opts, const stab_path_choice *choice,
                       stab_ctx **out);

}  // namespace stab
