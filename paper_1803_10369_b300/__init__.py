"""SRLA (arXiv 1803.10369) hot path on B300: CUDA kernels behind a C ABI (libsrla)."""
from .srla import (  # noqa: F401
    CARRIED,
    ENTRY_DTYPE,
    Group,
    NEW,
    SATURATED,
    Server,
    SUPER,
    Link,
    SRLAError,
    check_params,
    derived,
    lib,
    library_path,
    make_params,
    params_for,
    workspace_bytes,
)
