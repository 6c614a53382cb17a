"""GB300 (sm_103a) two-stage SCL + MP-WSD decoder: the libmpwsd C ABI and its
Python binding. Build the shared library with ``paper_2602_08501_gb300.build``."""
from .mpwsd import (  # noqa: F401
    Code,
    MpwsdError,
    Pool,
    Workspace,
    declared_symbols,
    enumerate_codewords,
    lib,
    rm_frozen,
)
