"""GB300-native k-d tree queries: find-closest-point and k-nearest-neighbour
search over left-balanced, complete, level-order k-d trees with the
stack-free (curr, prev) traversal of Wald, arXiv 2210.12859.

The compute path is the CUDA library ``libkdt.so`` (C ABI in include/kdt.h);
``paper_2210_12859_gb300.kdt`` is its Python binding.  It is imported lazily
so that the input generators in ``synth`` work without the library.
"""


def __getattr__(name):
    if name == "kdt":
        import importlib

        return importlib.import_module(".kdt", __name__)
    raise AttributeError(name)
