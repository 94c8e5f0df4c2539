"""Processor type ids and per-type parameter widths (fixed data, no arithmetic).

Type letters follow the paper (Sec. 2 Fig. 1 legend, Fig. 2b legend): i input,
o output, m mix, g gain/panning, s stereo imager, e equalizer, c compressor,
d multitap delay, r reverb, n noisegate; the multi-port processors (Eq. 1a with M, N
> 1) are p split, j merge and k sidechain compressor.

Parameter widths N_t (the columns of P[t], Sec. 2 "Graph representations"):
  g: 2   ln-gain per channel (Eq. 2)
  s: 1   ln side gain (Eq. 3)
  e: 8   band gains in dB (8-band design of the zero-phase FIR, Eq. 4)
  c: 4   [alpha, T, W, R]; T and W in natural-log energy units (Eq. 8-12)
  d: 176 2 channels x 4 taps x [Re z, Im z, 20 ln-magnitudes] (Eq. 14-15)
  r: 50  [mid, side] x [H0, H_delta] x 12 bands (ln-magnitude), then q_dry, q_wet
  n: 4   [alpha, T, W, R] like the compressor, with the gate curve (Eq. 13)
  p: 0   split (1 input, 2 outputs: mid, side)
  j: 0   merge (2 inputs: mid, side; 1 output)
  k: 4   sidechain compressor (2 inputs: main, key) [alpha, T, W, R] as the compressor
  a: 5   compressor with attack/release ballistics [alpha_attack, alpha_release, T, W, R]

Widths of the paper's own processor settings (Sec. 3), ``PAPER_PARAM_COLS``:
  e: 1024 ln-magnitudes of the 2047-tap zero-phase FIR
  d: 880  2 channels x 20 taps (one per 100 ms slot) x [Re z, Im z, 20 ln-magnitudes]
  r: 768  [mid, side] x [H0, H_delta] x 192 ln-magnitudes (STFT 384 / hop 192)
"""
I, O, M, G, S, E, C, D, R, N, P, J, K, A = range(14)
TYPE_LETTERS = "iomgsecdrnpjka"
TYPE_IDS = {ch: k for k, ch in enumerate(TYPE_LETTERS)}
PARAM_COLS = {I: 0, O: 0, M: 0, G: 2, S: 1, E: 8, C: 4, D: 176, R: 50, N: 4, P: 0, J: 0, K: 4, A: 5}
PAPER_PARAM_COLS = dict(PARAM_COLS)
PAPER_PARAM_COLS.update({E: 1024, D: 880, R: 768})


def param_cols(preset="compact"):
    """Parameter widths per type for a processor preset ("compact" or "paper")."""
    if preset not in ("compact", "paper"):
        raise ValueError(preset)
    return PAPER_PARAM_COLS if preset == "paper" else PARAM_COLS
