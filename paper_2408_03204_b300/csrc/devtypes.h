// Plain structs shared by the host planner and the device kernels (same layout on both).
#pragma once
#include <stdint.h>

namespace grafx {

enum NodeKind : int16_t { KIND_INPUT = 0, KIND_OUTPUT = 1, KIND_INTERNAL = 2 };

// One node in reordered (new-id) order.  A node's output row Y_v lives in one of
// three buffers chosen by `kind` (sources for inputs, the caller's out buffer for
// outputs, the workspace U region otherwise); likewise its adjoint row.
struct alignas(16) NodeDev {
  int64_t off_y;   // float offset of the [2][pitch] output row inside its buffer
  int64_t off_a;   // float offset of the [2][pitch] adjoint row inside its buffer
  int32_t len;     // signal length L of the node's graph
  int32_t pitch;   // channel stride (L rounded up to a multiple of 4)
  int32_t prow;    // row of P[type] read by the node (I^P of Algorithm 1)
  int16_t kind;    // NodeKind
  int16_t type;    // GRAFX_T_*
  int32_t grow;    // row of the gradient table the backward writes: prow, or with a
                   // source batch the node's own row of the per-copy gradient table
  int32_t rstride; // floats between the node's consecutive port rows (output port k at
                   // off_y + k rstride, input-port adjoint l at off_a + l rstride)
  int32_t pad[2];
};

// Row reference of a CSR entry: the buffer (NodeKind) in the top bits, the float offset
// of the row inside it below.
constexpr int REF_SHIFT = 60;
constexpr int64_t REF_MASK = (int64_t(1) << REF_SHIFT) - 1;

struct alignas(16) int4_ { int32_t x, y, z, w; };
struct alignas(8) int2_ { int32_t x, y; };
struct alignas(8) float2_ { float x, y; };

// One output row of the loss.
struct alignas(16) LossRow {
  int64_t off;            // float offset of the row in out / target / d_out
  int64_t frame_off[3];   // float offset of the row's frame buffer per resolution
  int64_t spec_off[3];    // float2 offset of the row's spectra per resolution: planes
                          // Y_l, Y_r, (|T_l|, |T_r|) of [frames][M/2+1] each
  int32_t len, pitch;
  int32_t n_frames[3];
  int32_t group_off[3];   // first partial-statistics group of the row per resolution
  int32_t n_groups[3];
  int32_t pad;
};

constexpr int TWIDDLE_N = 8192;   // twiddle table size: exp(-2 pi i m / 8192)
constexpr int EW_TILE = 4096;     // samples per elementwise work item (4 float4 per thread and channel)
constexpr int N_RES = 3;          // loss resolutions 512, 1024, 2048

// multitap delay (Eq. 14-15).  Compact layout: 4 taps per channel, each anywhere in
// [0, N_d), N_d = 32768.  Slot layout (the paper's): 20 taps per channel, tap m in
// [m S, m S + S) with the surrogate of length N_d = S = fs / 10.  The tap count, N_d,
// the slot width and the lag partitions are runtime values of the plan (DevCtx).
constexpr int DL_NFFT = 32768;     // compact surrogate transform length N_d
constexpr int DL_TAPS = 4;         // compact taps per channel
constexpr int DL_SLOT_TAPS = 20;   // slot-layout taps per channel (2 s in 100 ms slots)
constexpr int DL_FIR = 39;         // zero-phase FIR per tap (20 log-magnitudes)
constexpr int DL_K = (DL_FIR + 1) / 2;
constexpr int DL_ROW = 2 + DL_K;   // parameters per (channel, tap): Re z, Im z, 20 log-magnitudes
constexpr int DL_TILE = 2048;      // outputs per forward / adjoint work item
constexpr int DL_B = 4096;         // block of the lag correlation
constexpr int DL_M = 2 * DL_B;     // its FFT size
constexpr int DL_PMAX = 32;        // lag partitions: lags [-B, (P-1) B) cover [-19, reach + 19)
constexpr int DL_CHUNK = 32;       // bins per accumulation work item
constexpr int DL_MAX_BLOCKS = 128; // signals with delay nodes: at most 2^19 samples

// filtered-noise reverb (Eq. 6-7).  Compact layout: STFT 1024 / hop 256, 12 bands,
// dry and wet gains.  Paper layout: STFT 384 / hop 192, 192 per-bin log-magnitudes
// per filter, wet only.  The STFT size, hop and frame count are runtime values.
constexpr int RV_LEN = 88200;      // impulse response: 2 s at 44.1 kHz
constexpr int RV_N = 1024;         // compact STFT size
constexpr int RV_HOP = 256;
constexpr int RV_F = 1 + RV_LEN / RV_HOP;              // 345 centred frames
constexpr int RV_BINS = RV_N / 2 + 1;
constexpr int RV_BANDS = 12;
constexpr int RV_COLS = 50;        // [mid, side] x [H0, Hd] x 12 bands, q_dry, q_wet
constexpr int RV_PN = 384;         // paper STFT size
constexpr int RV_PHOP = 192;
constexpr int RV_P = (RV_LEN + DL_B - 1) / DL_B;       // 22 partitions of 4096 taps
constexpr int RV_HLEN = RV_P * DL_B;

// status bits written by kernels
constexpr uint32_t ST_TIMEOUT = 1u;
constexpr uint32_t ST_BOUNDS = 2u;

}  // namespace grafx
