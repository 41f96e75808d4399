"""LIDER batched query search on one B300 (sm_103a).

The CUDA library (``liblider.so``) is loaded by ``paper_2205_00970_b300.lider``;
importing the package itself loads nothing, so the seeded input generators in
``synth`` can be used without a GPU.
"""
