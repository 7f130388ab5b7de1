"""B300-native hp-version time-stepping spectral Monte Carlo (sm_103a).

The CUDA library (libspmc.so, C-ABI in include/spmc.h) runs every step of the
method; ``Plan`` is its Python front end over PyTorch device memory.
``workloads`` holds the seeded synthetic inputs.
"""
__all__ = ["Plan", "workloads"]


def __getattr__(name):
    if name == "Plan":
        from .api import Plan
        return Plan
    raise AttributeError(name)
