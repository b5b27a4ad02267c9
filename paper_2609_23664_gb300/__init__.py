"""GB300-native engine for workload-level reuse of shared circuit prefixes.

The native library (libquwarp.so, sm_103a) is loaded lazily by
`paper_2609_23664_gb300.quwarp`; importing the package itself loads nothing.
"""
__all__ = ["workloads", "quwarp"]
