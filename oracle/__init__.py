"""CPU FP64 oracle of the PHSVDS method (arXiv 1408.5535).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` may import this package; the product path
(the CUDA library and its Python binding) never does.  It shares no code with
the GPU path.
"""
