// Internal definitions shared by the host runtime (koma_runtime.cpp) and the
// CUDA kernels (koma_kernels.cu). Not part of the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "koma.h"

namespace koma {

// ---------------------------------------------------------------------------
// Step records: the discretised sequence after host preprocessing.
//
// The kernel keeps, per spin, the magnetisation at a reference time t_ref
// (the end of the last RF step, or t_0). Between RF steps the state is never
// stepped: precession + relaxation over any interval is the closed form of
// the per-step updates (the product of the per-step e^{i phi} and decay
// factors; Eq. Rotation_precession with the integral phase of the
// sequence-aware time stepping section, and the relaxation update):
//   Mxy(t) = Mxy(t_ref) e^{-tau/T2} e^{-i 2 pi (K(t).x + df tau)}
//   Mz(t)  = M0 + (Mz(t_ref) - M0) e^{-tau/T1}
// with tau = t - t_ref, df = dw / 2 pi (Hz) and K(t) = gammabar * integral of
// G from t_ref to t (turns/m, trapezoid rule over the gradient vertices,
// exact for piecewise-linear G). K and tau are accumulated on the host in
// FP64 and stored as hi/lo FP32 pairs.
// ---------------------------------------------------------------------------

enum RecType : int32_t {
    REC_RF = 0,     // one excitation step: rotate about the step's field, relax
    REC_PREC = 1,   // move t_ref: materialise the state at (K, tau), then K = tau = 0
    REC_ADC = 2,    // `count` samples at (K0 + l dK, tau0 + l dtau), l < count
    REC_MAP = 3,    // a repeated pulse as a whole: apply map k0 (compacted streams only)
};

// largest number of samples in one ADC record (the recurrence between exact
// evaluations never runs longer than this)
constexpr int kMaxAdcRun = 128;
constexpr int kCountMask = 0xffff;   // samples field of an ADC record's count
// Device status word bits (koma_sync reads and clears them): 1 = a bounded
// wait of a kernel gave up; 2 = the bounded-wait self-check gave up (as it
// is meant to); the others: a record pointed outside its launch's buffers
// and its access was skipped: 4 = an ADC run past n_adc or before the
// samples already staged, 8 = a map slot, 16 = a readout snapshot row,
// 32 = a tensor-core readout run.
constexpr int kStatusTimeout = 1;
constexpr int kStatusWaitCheck = 2;
constexpr int kStatusBadAdc = 4;
constexpr int kStatusBadMap = 8;
constexpr int kStatusBadSnap = 16;
constexpr int kStatusBadRun = 32;
constexpr int kTermShift = 16;       // nonzero-term bits of PREC/ADC records

// Matrix form of the readout. ADC runs whose samples share the per-sample
// rotator (the same dK and dtau, as FP32 values) are grouped, up to kMmaRuns
// runs a group. Sample l of run r sums E_s(r) z_s^l over the spins s, with
// E_s(r) the spin's transverse magnetisation at the run's first sample and
// z_s the rotator e^{-dtau/T2} e^{-i 2 pi (dK.x + df dtau)}: a complex matrix
// product C[r][l] = sum_s E_s(r) z_s^l over spins, taken on the tensor cores.
// E_s(r) = Mxy_s(t_ref) e^{-tau0/T2} e^{-i 2 pi (K0.x + df tau0)} is
// evaluated there too, from the run's (K0, tau0) and a snapshot of
// Mxy(t_ref): the state is constant between RF and PREC records, so the
// Bloch kernel stores one snapshot per such stretch ("block") that holds
// matrix-form runs, at the block's first flagged record (kMmaSnapFlag), into
// row `snap` of an [n_snaps][n_pad] buffer (rows in record order), and
// steps no flagged sample itself.
constexpr int kMmaRuns = 64;          // runs per group: 128 matrix rows (Re, Im of each)
constexpr int kMmaFlag = 1 << 28;     // ADC record count bit: sampled by the matrix form
constexpr int kMmaSnapFlag = 1 << 29; // ... and the first of its block: store the snapshot
constexpr int kMmaMinRuns = 8;        // smallest group worth a tensor-core pass
constexpr int64_t kMmaMinSamples = 1024;

struct MmaGroup {
    float dk[3];      // rotator: dK (turns/m) ...
    float dtau;       // ... and dtau (s), as in the group's records
    int32_t run0;     // first entry of the group in the run table
    int32_t n_runs;   // 1..kMmaRuns
    int32_t max_len;  // longest run (samples)
    int32_t one_snap; // 1: every run of the group uses the same snapshot row
};
static_assert(sizeof(MmaGroup) == 32, "MmaGroup layout");
struct MmaRun {
    int64_t k0;       // first sample
    int32_t len;      // samples
    int32_t snap;     // snapshot row of the run's block
    float kh[3], kl[3];  // K0 (turns/m) hi/lo, relative to the block's t_ref
    float th, tl;     // tau0 (s) hi/lo
    int32_t pad_[4];
};
static_assert(sizeof(MmaRun) == 64, "MmaRun layout");

// Repeated RF pulses. Every RF step maps the magnetisation affinely
// (rotation about the step's constant field, then relaxation: M -> D R M + b
// with D = diag(E2, E2, E1) and b = (0, 0, M0 (1 - E1))), so a whole run of
// RF steps does too: M -> A M + c with A = D_N R_N ... D_1 R_1 and c the
// run's response to M = 0 (the composition of the per-step updates of Eq.
// Rot_exc and the relaxation equations, in exact arithmetic the same result
// as stepping). A run of RF records that recurs unchanged (the same pulse
// under the same gradient: the excitation and refocusing pulses of every
// shot of a multi-shot sequence) gets a map slot: a pre-pass kernel computes
// (A, c) per spin from the steps of the pulse, and the FP32 Bloch kernel
// applies it at every occurrence instead of stepping the run. In the full
// record stream the run's header carries k0 = 1 + slot (0: stepped); the
// kernels that apply maps walk a compacted stream in which every such run is
// one REC_MAP record (k0 = slot, count = the run's length).
constexpr int kMaxRfMaps = 8;
constexpr int kRfMapFloats = 12;     // per spin and map: three float4 rows (A_i0, A_i1, A_i2, c_i)
constexpr int kRfMapMinRuns = 3;     // occurrences that make a map worth its pre-pass
constexpr int kRfMapMinLen = 4;      // RF steps of a run worth a map
struct RfMapPulse {
    int64_t rec_begin;  // header record of the pulse's first occurrence
    int32_t len;        // RF records of the run
    int32_t pad_;
};
static_assert(sizeof(RfMapPulse) == 16, "RfMapPulse layout");

// 64-byte record of the FP32 split-phase path.
//   RF:   a[0..2] pi gbar gammabar dt (rad/m)   a[3..4] pi B1 gammabar dt (rad):
//         the half-angle rotation vector of the step's field
//         a[5]    |a[3..4]|^2             a[6] dt (s)
//         The first record of every run of consecutive RF records carries the
//         run's length in `count` and the run's maxima in a[7] |a[3..4]|,
//         a[8..10] |a[d]|, a[11] dt; later ones have count 0.
//   PREC: a[0..5] Kx hi,lo Ky hi,lo Kz hi,lo (turns/m)   a[6..7] tau hi,lo (s)
//   ADC:  a[0..7] K0, tau0 as in PREC     a[8..10] dK (turns/m)   a[11] dtau (s)
//   PREC/ADC: count = samples (ADC; low 16 bits) | nonzero-term bits << 16
//         (bit 0 Kx, 1 Ky, 2 Kz, 3 tau), so the kernel skips zero phase terms
//         without testing the payload.
//   RF header records: k0 = 1 + the run's map slot when the run is a repeated
//         pulse taken by its map, else 0.
//   MAP:  (compacted streams) k0 = map slot, count = RF steps it stands for.
struct alignas(16) Rec32 {
    int32_t type;
    int32_t count;
    int64_t k0;     // ADC: index of the first sample
    float a[12];
};
static_assert(sizeof(Rec32) == 64, "Rec32 must be 64 bytes");

// Motion (the phantom's u(x, t) as a constant velocity, x(t) = x + v t, t
// from t_0): the phase from t_ref to t becomes
//   2 pi (K.x + K1.v + df tau),  K1 = gammabar * integral from t_ref to t of G(s) s ds
// (turns s/m; s is absolute time, trapezoid-exact per step for linear G).
// Within an ADC run of uniformly spaced samples under a gradient that
// repeats from one sample interval to the next (a constant readout
// gradient), the K1 increment of interval l is dK1_0 + l dtau dK, so the
// per-sample phase increment grows linearly in l. The host only joins
// samples into a run when their K1 increments follow that rule.

// 128-byte record of the FP64 path (same meaning, FP64 values, no hi/lo).
//   RF:   a[0..2] gbar*gammabar*dt  a[3..4] B1*gammabar*dt  a[5] dt
//         a[6] t_mid (s): the step's midpoint, where a moving spin sits
//   PREC: a[0..2] K  a[3] tau  a[4..6] K1
//   ADC:  a[0..2] K0 a[3] tau0  a[4..6] dK  a[7] dtau  a[8..10] K1 of the
//         first sample  a[11..13] dK1_0 (K1 increment to the second sample)
struct alignas(16) Rec64 {
    int32_t type;
    int32_t count;
    int64_t k0;
    double a[14];
};
static_assert(sizeof(Rec64) == 128, "Rec64 must be 128 bytes");

// 128-byte record of the FP32 motion kernel: Rec32's fields in a[0..11]
// (same meaning, run headers included) plus
//   RF:   a[12] max t_mid over the RF run (header only)   a[13] t_mid (s)
//   PREC: a[8..13] K1 x, y, z hi/lo
//   ADC:  a[12..17] K1 hi/lo of the first sample   a[18..23] dK1_0 hi/lo
//   PREC/ADC term bits: bits 0..3 as Rec32, bits 4..6 K1 x, y, z nonzero.
struct alignas(16) RecM {
    int32_t type;
    int32_t count;
    int64_t k0;
    float a[28];
};
static_assert(sizeof(RecM) == 128, "RecM must be 128 bytes");

// Per-spin device layout: structure of arrays, each array n_pad long.
enum P32 : int {
    P32_XH = 0, P32_XL, P32_YH, P32_YL, P32_ZH, P32_ZL,
    P32_FH, P32_FL,   // df = dw / 2 pi, Hz, hi/lo
    P32_M0,
    P32_R1, P32_R2,   // log2(e) / T1, log2(e) / T2 (0 for +inf)
    P32_N
};
enum P64 : int {
    P64_X = 0, P64_Y, P64_Z,
    P64_F,            // df, Hz
    P64_T1, P64_T2,   // s (+inf allowed)
    P64_M0,
    P64_N
};
// Velocities of a moving phantom: FP32 hi/lo block [PV32_N][n_pad] and FP64
// block [3][n_pad] (m/s).
enum PV32 : int { PV32_XH = 0, PV32_XL, PV32_YH, PV32_YL, PV32_ZH, PV32_ZL, PV32_N };

struct BlochLaunch {
    int grid = 0;
    int block = 0;
    int spins_per_thread = 0;
    int64_t spins_per_cta = 0;
};

struct BlochArgs {
    const float* p32 = nullptr;     // [P32_N][n_pad]
    const double* p64 = nullptr;    // [P64_N][n_pad]
    int64_t n_pad = 0;
    int64_t n = 0;
    const int64_t* cta_begin = nullptr;  // [spin CTAs + 1] first spin of each (grouped), or null
    int64_t spins_per_cta = 0;           // uniform split when cta_begin is null
    // ADC-run split (FP32 Bloch and motion kernels): `split` CTAs walk each
    // spin range; CTA spin_cta * split + p takes the ADC records whose index
    // is p mod split and writes those samples of the range's partial row
    // (one row per spin range, every sample written by exactly one part; all
    // parts step every RF and PREC record). For launches whose spins fill
    // few warps. 1 = off.
    const void* rec = nullptr;
    int64_t n_rec = 0;
    void* partial = nullptr;        // FP32: float2 [grid][n_adc]; FP64: double2 [grid][n_adc]
    int64_t n_adc = 0;
    int* status = nullptr;          // device flag word (bit 0: a bounded wait gave up)
    int split = 1;
    float ext[4] = {0, 0, 0, 0};    // max |x|, |y|, |z| (m), |df| (Hz) over the phantom
    int used = 0;                   // bit d: coordinate d (x, y, z, df) is nonzero somewhere;
                                    // bit 4 + d: velocity component d is nonzero somewhere
    // moving phantoms (motion kernels only)
    const float* pv32 = nullptr;    // [PV32_N][n_pad]
    const double* pv64 = nullptr;   // [3][n_pad]
    float vext[3] = {0, 0, 0};      // max |v_x|, |v_y|, |v_z| (m/s)
    // matrix-form readout (FP32 static kernel only): if set, ADC records
    // carrying kMmaFlag are not sampled here; those also carrying
    // kMmaSnapFlag store Mxy(t_ref) x mma_escale into the next row of this
    // [n_snaps][n_pad] buffer (rows in record order)
    float2* mma_snap = nullptr;
    float mma_escale = 1.f;         // power of two keeping E in FP16 range
    // repeated RF pulses (FP32 static kernel only): `rec` is then the
    // compacted stream, whose REC_MAP records apply map k0 of this
    // [n_rf_maps][3][n_pad] float4 buffer (row i of A and c_i per spin)
    const float* rf_maps = nullptr;
    int n_rf_maps = 0;
    int64_t n_mma_snaps = 0;        // rows of mma_snap
};

// Pre-pass of the repeated-pulse maps: for every spin j < n and pulse p,
// (A, c) of pulse p's RF records into maps[p], three float4 rows per spin (row i of A, c_i).
struct RfMapArgs {
    const float* p32 = nullptr;
    int64_t n_pad = 0;
    int64_t n = 0;
    const Rec32* rec = nullptr;
    const RfMapPulse* pulses = nullptr;
    int n_pulses = 0;
    float* maps = nullptr;          // [n_pulses][3][n_pad] float4: row i of A, then c_i
    float ext[4] = {0, 0, 0, 0};
};

// Tensor-core readout (K6): CTA c takes spins [c spins_per_cta, +spins_per_cta)
// in blocks of 32 and, for every group, writes the group's samples of row c
// of `partial` (float2 [grid][n_adc]).
struct MmaArgs {
    const float* p32 = nullptr;
    int64_t n_pad = 0;
    int64_t n = 0;
    const float2* snap = nullptr;    // [n_snaps][n_pad] Mxy(t_ref) of each block, scaled by 1 / einv
    int used = 0;                    // bit d: coordinate d (x, y, z, df) nonzero somewhere
    const MmaGroup* groups = nullptr;
    int32_t n_groups = 0;
    const MmaRun* runs = nullptr;
    float2* partial = nullptr;
    int64_t n_adc = 0;
    int64_t spins_per_cta = 0;       // multiple of 32
    float einv = 1.f;                // 1 / the power-of-two scale E was stored with
    int* status = nullptr;
};

struct ItemArgs {
    const float* p32 = nullptr;
    const double* p64 = nullptr;
    int64_t n_pad = 0;
    const int64_t* item_begin = nullptr;  // [n_items + 1] first spin of each item
    const int32_t* order = nullptr;       // [n_items] processing order (longest first)
    int64_t n_items = 0;
    int* counter = nullptr;               // batch counter, zero at launch
    const void* rec = nullptr;            // Rec32 records
    int64_t n_rec = 0;
    void* partial = nullptr;              // float2 [n_items][n_adc]
    int64_t n_adc = 0;
    int* status = nullptr;
    float ext[4] = {0, 0, 0, 0};
    int used = 0;
    int uni_relax = 0;                    // every group has one T1 and one T2 (relaxation once per thread)
    // K3z: units of up to 8 consecutive spins of one group, packed across
    // groups (a warp takes 32 consecutive units); each (warp, group) segment
    // is one item, i.e. one partial row
    const int64_t* unit_begin = nullptr;  // [n_units + 1] first spin of each unit
    const int32_t* unit_item = nullptr;   // [n_units] item of each unit
    int64_t n_units = 0;
};

struct ReduceArgs {
    const void* partial = nullptr;
    int grid = 0;                       // CTAs that wrote partial rows
    const int32_t* group_cta = nullptr; // [n_groups + 1] CTA range of each group (null: one group)
    int64_t n_groups = 1;
    int64_t n_adc = 0;
    double* sig = nullptr;              // [n_groups][n_adc][2]
    // samples k with from_mma[k] != 0 come from the tensor-core readout's
    // rows instead (one group only)
    const void* partial_mma = nullptr;
    int grid_mma = 0;
    const uint8_t* from_mma = nullptr;
};

// One batch of the serving kernel: a spin range of one request's phantom,
// walked through that request's records; warp w of the batch takes spins
// [spin_begin + 32 S w, +32 S) and writes row w (rows + w * n_adc).
struct BatchDesc {
    const float* p32;
    int64_t n_pad;
    const Rec32* rec;
    int64_t n_rec;
    float2* rows;
    int64_t n_adc;
    int64_t spin_begin, spin_end;
    int64_t rec_begin, rec_end;  // records walked by this launch
    float* state;                // [3][n_pad] checkpoint between chunks (null: one chunk)
    float ext[4];
    int used;
    int n_rf_maps;               // map slots of the request's repeated pulses (0: none)
    int64_t rf_hdr;              // header of the RF run rec_begin lies inside (-1: none)
    const float* rf_maps;        // [n_rf_maps][3][n_pad] float4 (row of A, c); `rec` is then compacted
};
static_assert(sizeof(BatchDesc) == 128, "BatchDesc layout");

struct BatchArgs {
    const BatchDesc* desc = nullptr;
    const int64_t* n_batches_dev = nullptr;  // device: batches in the table
    int* counter = nullptr;                  // batch counter, zero at launch
    int* status = nullptr;
};

// Host preprocessing (koma_runtime.cpp), shared with the server: validate a
// phantom and build its FP32 device block [P32_N][n_pad] and extents (max
// |x|, |y|, |z|, |df|); validate a sequence and build its FP32 records.
// Return a koma_status; `err` gets the message.
int host_phantom32(int64_t n, const double* x, const double* y, const double* z, const double* pd,
                   const double* t1, const double* t2, const double* dw, std::vector<float>& h32, int64_t& n_pad,
                   double (&max_abs)[4], std::string& err);
int host_records32(int64_t n_steps, const double* dt, const double* gx, const double* gy, const double* gz,
                   const double* b1_re, const double* b1_im, const uint8_t* adc, std::vector<Rec32>& r32,
                   koma_sequence_info& info, std::string& err);
// The upload's input rules alone, without building anything (requests the
// server hands to koma_simulate, which converts on the device): spins
// (finite, pd >= 0, T1/T2 > 0 or +inf) and sequence arrays (dt > 0 finite,
// finite G and B1, adc 0/1). `info` receives n_steps, n_adc, n_rf and, in
// n_materialize, the number of RF runs (the state changes only there, so the
// readout keeps at most that many + 1 snapshots).
int host_check_phantom(int64_t n, const double* x, const double* y, const double* z, const double* pd,
                       const double* t1, const double* t2, const double* dw, std::string& err);
int host_check_sequence(int64_t n_steps, const double* dt, const double* gx, const double* gy, const double* gz,
                        const double* b1_re, const double* b1_im, const uint8_t* adc, koma_sequence_info& info,
                        std::string& err);
// Repeated RF pulses of a record stream: marks the header records of the
// runs taken by maps (k0 = 1 + slot) and returns the slots' pulses; `info`
// gets the n_rf_map* counts.
void host_rf_maps32(std::vector<Rec32>& r32, std::vector<RfMapPulse>& pulses, koma_sequence_info& info);
// The compacted stream of a marked one: every run taken by a map becomes
// one REC_MAP record; everything else is copied.
void compact_records32(const std::vector<Rec32>& r32, std::vector<Rec32>& out);

// Launch helpers (koma_kernels.cu). Return a cudaError_t as int.
// Phantom conversion: p64 [P64_N][n_pad] holds the raw rows x, y, z, dw
// (rad/s), T1, T2, pd for spins j < n; writes the FP32 block p32
// [P32_N][n_pad], replaces row P64_F by df = dw / 2 pi and fills the padding
// (inert spins: zero state, T1 = T2 = 1 in the FP64 block). It also checks
// every spin (the upload's input rules) and takes the extents: `cs` must hold
// first_bad = ~0 and max_bits = 0 before the launch; afterwards first_bad
// is the lowest invalid spin (~0: none) and max_bits the bit patterns of
// max |x|, |y|, |z| (m), |df| (Hz) and pd over the spins.
struct ConvertStatus {
    unsigned long long first_bad;
    unsigned long long max_bits[5];  // and max pd
};
int launch_phantom_convert(double* p64, float* p32, int64_t n, int64_t n_pad, ConvertStatus* cs, void* stream);
int launch_bloch_fp32(const BlochArgs& a, const BlochLaunch& L, void* stream);
int launch_bloch_fp64(const BlochArgs& a, const BlochLaunch& L, void* stream);
// Moving phantoms: FP32 motion kernel (RecM records, 2 spins per thread) and
// the FP64 kernel's motion variant (Rec64 records with K1).
int launch_bloch_motion(const BlochArgs& a, const BlochLaunch& L, void* stream);
int launch_bloch_fp64_motion(const BlochArgs& a, const BlochLaunch& L, void* stream);
int motion_ctas_per_sm(int block);
// Tensor-core readout: `grid` CTAs of the kernel's fixed shape (one per SM).
int launch_readout_mma(const MmaArgs& a, int grid, void* stream);
// Repeated-pulse maps (one launch for all pulses).
int launch_rf_maps(const RfMapArgs& a, void* stream);
constexpr int kMotionSpinsPerThread = 2;
int launch_reduce(const ReduceArgs& r, bool fp64_partials, void* stream);
// One thread waits, bounded by limit_ns, on an mbarrier nothing completes,
// then sets bit 1 of *status (the timeout path of the record-tile waits).
int launch_bounded_wait_check(int* status, unsigned long long limit_ns, void* stream);
// `tile`: step records per shared-memory tile, 64, 128 or 256.
int launch_items(const ItemArgs& a, int grid, int block, int spins_per_thread, int tile, void* stream);
int items_ctas_per_sm(int spins_per_thread, int block, int tile);
// K3z, the grouped kernel for dictionaries of isochromats along z (spins
// differ only in z, one T1/T2 per group, RF without z gradient, one sample
// per ADC record): one unit of up to 8 spins per thread (a.unit_begin,
// a.unit_item, a.n_units); `tile` 128 or 256 records. `a.rec` is the
// K3z copy of the stream (RF records with the rotation in a[0..3], PREC/ADC
// records with -2 pi Kz in a[8]); `small_phase`: |z Kz| <= 1 turn for every
// spin and record, the phase as one FP32 product (then block <= 128).
int launch_items_z(const ItemArgs& a, int grid, int block, int tile, bool small_phase, void* stream);
int items_z_ctas_per_sm(int block, int tile, bool small_phase);
// Serving kernel (4 spins per thread, `block` threads: a batch is 128 x
// block/32 spins).
int launch_batches(const BatchArgs& a, int grid, int block, void* stream);
int batches_ctas_per_sm(int block);
// Static partial-sum scratch of koma_simulate_static: capacity in float2
// elements, and its device address on `device` (which must be current; the
// address is looked up once per device and cached).
size_t static_partials_capacity();
int static_partials_ptr(int device, void** out);
// Largest block size the FP32 / FP64 Bloch kernels accept, and their
// resident CTAs per SM at that size.
int bloch_max_block();
int bloch_ctas_per_sm(bool fp64, int spins_per_thread, int block);

}  // namespace koma
