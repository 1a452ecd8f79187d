"""GB300 (sm_103a) implementation of the hot path of PLAST's bank-to-bank
protein comparison (Nguyen & Lavenier, INRIA RR-6513, 2008): subset-seed
indexing (stage 0), all-pairs ungapped extension per shared key (stages 1-2)
and the banded small gapped extension of the survivors (stage 3.1), plus the
six-frame translation of TPLAST-N.

The C ABI is include/plast.h (libplast.so, built by ``build.build()``);
``binding`` exposes it to Python under the same names.  ``synth`` draws the
seeded synthetic banks.  Submodules are imported on first use so that
``synth`` can be used without a GPU or torch.
"""
import importlib

__all__ = ["binding", "build", "synth"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
