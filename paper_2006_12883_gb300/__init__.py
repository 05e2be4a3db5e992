"""GB300 (sm_103a) space-time multigrid / SDC library for reaction-diffusion
problems discretised by right-Radau collocation in time (Benedusi, Minion,
Krause, arXiv 2006.12883).  The compute path is libst.so (include/st.h);
``stlib`` is its ctypes binding and ``autograd`` the torch.autograd wrapper.
"""
from .build import build  # noqa: F401
