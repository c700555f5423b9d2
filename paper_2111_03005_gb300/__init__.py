"""GB300-native global switch round of the Global Edge Switching Markov Chain.

The compute path is the C-ABI library ``libgesmc.so`` (hand-written CUDA for
sm_103a, built from ``csrc/``); ``gesmc`` is its thin ctypes binding and
``inputs`` makes seeded synthetic starting graphs.
"""
