"""GB300-native (sm_103a) trapped-ion timestep: all-pairs Coulomb + linear Paul trap +
Langevin bath + velocity Verlet, behind the C ABI of libiontrap.so (include/iontrap.h).

The Python names are those of the C entry points (see ``native``).  The first access to
any of them loads libiontrap.so and raises ImportError if it has not been built; the
``build`` submodule is importable without the library.
"""
import importlib


def __getattr__(name):
    if name.startswith("__"):
        raise AttributeError(name)
    if name in ("build", "native"):
        return importlib.import_module("." + name, __name__)
    native = importlib.import_module(".native", __name__)
    try:
        return getattr(native, name)
    except AttributeError:
        raise AttributeError(f"module {__name__!r} has no attribute {name!r}") from None


def __dir__():
    native = importlib.import_module(".native", __name__)
    return sorted(set(globals()) | set(dir(native)))
