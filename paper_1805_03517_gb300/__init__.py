"""GB300-native Flow Fields dense matching (the matching stage of FlowFields++, arXiv 1805.03517, Sec. 3.1).

* ``paper_1805_03517_gb300.ff``      -- binding of the C-ABI library libff.so (include/ff.h) and ``Matcher``
* ``paper_1805_03517_gb300.build``   -- builds libff.so in-tree for sm_103a
* ``paper_1805_03517_gb300.synth``   -- seeded synthetic KITTI-/Sintel-shaped frame pairs
* ``paper_1805_03517_gb300.configs`` -- the matching workloads and parameters

Importing the package loads nothing native; ``ff.lib()`` loads libff.so and fails loudly if it is missing.
"""
