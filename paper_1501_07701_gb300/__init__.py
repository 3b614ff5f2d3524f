"""Bulk MTGP32 generation on GB300 (sm_103a).

The CUDA library is ``libmtgp.so`` (C ABI in ``include/mtgp.h``); its Python
binding is :mod:`paper_1501_07701_gb300.mtgp`.  Build with
:func:`paper_1501_07701_gb300.build.build`.
"""
