// Host-side helpers of the runtime (koma_runtime.cpp) used by the server:
// phantoms over device blocks the server already filled, and frees ordered
// on one stream. No kernel depends on this header.
#pragma once

#include <vector>

#include "koma.h"
#include "koma_internal.h"

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
// While one exists, the calling thread's host preprocessing runs serially
// (no worker pool): for threads that already run side by side, like the
// server's submitting and lane threads.
struct SerialHostScope {
    SerialHostScope();
    ~SerialHostScope();
    SerialHostScope(const SerialHostScope&) = delete;
    SerialHostScope& operator=(const SerialHostScope&) = delete;
    bool prev;
};
// A record stream seen as pointer and length: a builder's vector, or the
// records gathered straight into a staging buffer.
struct RecSpan {
    Rec32* p = nullptr;
    size_t n = 0;
    RecSpan() = default;
    RecSpan(Rec32* p_, size_t n_) : p(p_), n(n_) {}
    RecSpan(std::vector<Rec32>& v) : p(v.data()), n(v.size()) {}  // NOLINT: a view of the vector
    size_t size() const { return n; }
    Rec32& operator[](size_t i) const { return p[i]; }
    Rec32* begin() const { return p; }
    Rec32* end() const { return p + n; }
};
// compact_records32 writing into `out` (null: count only); returns the
// compacted stream's length.
size_t compact_records32_into(const Rec32* r32, size_t n, Rec32* out);
size_t compact_records32_into(const std::vector<Rec32>& r32, Rec32* out);
// koma_sequence_upload building the FP32 record stream only (for a
// simulation known to be FP32 on a static phantom).
koma_status sequence_upload_fp32(koma_ctx* ctx, int64_t n_steps, const double* dt, const double* gx,
                                 const double* gy, const double* gz, const double* b1_re, const double* b1_im,
                                 const uint8_t* adc, koma_sequence** out);

}  // namespace koma
