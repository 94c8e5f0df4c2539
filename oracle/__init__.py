"""FP64 CPU oracle for GRAFX graph rendering (arxiv 2408.03204).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
product path (``paper_2408_03204_b300``) never imports, calls or links anything
here, and this package imports nothing from the product path.

It is a plain, slow, obviously correct restatement of the paper:
  graph.py       graph checks, type schedules, node reordering, index maps
                 (Sec. 2 "Definitions", "Batched processing", "Type scheduling",
                 Algorithm 1, "Implementation details")
  processors.py  the processors and their analytic adjoints (Sec. 3, Eq. 2-15)
  render.py      one-node-at-a-time render in topological order, the scheduled
                 render of Algorithm 1, and the reverse-mode backward pass
  loss.py        multi-resolution STFT loss and its gradient
  optim.py       the parameter maps, Adam, and the delay z update of Sec. 3
                 "Multitap delay" (normalised gradient plus unit-circle penalty)
  warmstart.py   the warm-start network's features, forward and backward
Every floating-point step runs in float64; FP32 inputs are upcast exactly.

Parity unpinned (no closed form or brute force fixes them beyond the bounds
tested): the beam-search schedule between its optimal/greedy bounds; the weight
1e-2 of the delay's unit-circle penalty (the paper gives none; the penalty's form
and the normalisation are pinned by finite differences and scale invariance).
"""
