"""GB300-native B-char: mass-conserving ball-approximated characteristics
(Cheng & Droniou, arXiv 1908.05834) as a CUDA library behind a C ABI.

``paper_1908_05834_gb300.bchar`` is the ctypes binding of ``libbchar.so``;
``paper_1908_05834_gb300.inputs`` holds the seeded workload generators.
The binding is imported on first use so that the input generators can be used
without the compiled library.
"""
