"""B300-native DISC: demons CT->CBCT registration with simultaneous intensity correction.

The compute path lives in the CUDA library ``libdisc.so`` (sm_103a) behind the
C ABI of ``include/disc.h``; ``paper_1204_6295_b300.disc`` is its Python
binding.  ``paper_1204_6295_b300.phantom`` draws seeded synthetic inputs and
does not load the library.
"""

__all__ = ["disc", "phantom"]


def __getattr__(name):
    if name == "disc":
        import importlib
        return importlib.import_module(".disc", __name__)
    raise AttributeError(name)
