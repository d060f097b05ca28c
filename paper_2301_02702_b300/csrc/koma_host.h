// Host-side helpers of the runtime (koma_runtime.cpp) used by the server:
// phantoms over device blocks the server already filled, and frees ordered
// on one stream. No kernel depends on this header.
#pragma once

#include "koma.h"

namespace koma {

// A phantom of context `ctx` over device blocks the caller already filled
// and checked (p64 [P64_N][n_pad] as the conversion kernel leaves it, p32
// [P32_N][n_pad], the extents and max pd it reported). The blocks stay the
// caller's: the phantom's free leaves them alone, and they must outlive it.
int phantom_from_device(koma_ctx* ctx, int64_t n, double* p64, float* p32, const double (&max_abs)[4],
                        double max_pd, const int64_t* group_offsets, int64_t n_groups, bool uni_relax,
                        koma_phantom** out);
// Frees whose device blocks are released in order after the work already
// enqueued on `stream` (every use of the object was on that stream); no
// device-wide wait, unlike koma_phantom_free / koma_sequence_free.
void phantom_free_on(koma_phantom* ph, void* stream);
void sequence_free_on(koma_sequence* seq, void* stream);

}  // namespace koma
