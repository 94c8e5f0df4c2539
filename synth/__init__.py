"""Seeded synthetic workloads: mixing graphs, source signals and processor parameters.

This package is shared by the FP64 oracle (``oracle/``) and the CUDA path
(``paper_2408_03204_b300``).  It holds none of the rendering method's arithmetic:
no scheduling, no reordering, no processor maths.  It only draws random graphs,
random physical parameters and random source audio from numpy PCG64 streams, so
that both sides receive bit-identical FP32 inputs.

Node type ids are fixed data (the paper's type letters, Sec. 2, Fig. 1 and 2b):
``i=0 o=1 m=2 g=3 s=4 e=5 c=6 d=7 r=8 n=9 p=10 j=11 k=12 a=13``.
"""
from .types import TYPE_IDS, TYPE_LETTERS, I, O, M, G, S, E, C, D, R, N, P, J, K, A, PARAM_COLS, PAPER_PARAM_COLS, param_cols  # noqa: F401
from .graphs import Graph, console_cfg1, console_cfg2, random_console, batch_cfg3, console_all_types  # noqa: F401
from .signals import sources, reverb_noise  # noqa: F401
from .params import random_params, neutral_params, union_params  # noqa: F401
