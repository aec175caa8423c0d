"""GB300-native TPC Time-Frame tracker (arxiv 2106.03636, synchronous TPC tracking).

``o2tpc`` is the ctypes binding of the C-ABI in ``include/o2tpc.h``;
``synth`` generates the seeded synthetic Time Frames.
"""
