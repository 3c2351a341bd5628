"""GB300-native engine for neutron histories with probability-conserved
cross-section biasing (arxiv 2304.06226).

The compute path is the CUDA library libtp.so (C ABI in include/tp.h); this
package builds it (`build`), binds it (`native`) and wraps it for PyTorch
(`engine`).  Importing `native` or `engine` requires the built library."""

__all__ = ["build", "native", "engine"]


def __getattr__(name):
    import importlib
    if name in __all__:
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
