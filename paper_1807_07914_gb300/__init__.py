"""GB300-native MPS simulation of parameterised circuits and Pauli-sum energies.

Importing the package loads nothing native. ``paper_1807_07914_gb300.tnmps``
is the thin ctypes binding of the C-ABI library ``libtnmps.so`` (built by
``paper_1807_07914_gb300.build``); ``paper_1807_07914_gb300.inputs`` builds the
seeded synthetic workloads.
"""
__all__ = ["inputs", "tnmps", "build"]
