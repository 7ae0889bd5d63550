"""GB300 (sm_103a) implementation of the symmetry-preserving JFNK hot path.

* ``jfnk``   ctypes binding of ``libjfnk.so`` (C ABI in ``include/jfnk.h``)
* ``build``  in-tree nvcc build of ``libjfnk.so``
* ``synth``  seeded synthetic workloads shaped like the paper's experiments
"""
