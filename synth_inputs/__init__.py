"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This package holds no arithmetic of the stencil-composition method: it only
draws random fields and evaluates the continuous manufactured solutions and
request traces that the workloads are defined by.  Both the CUDA path and the
CPU oracle receive their inputs from here.
"""
