"""Twofold summation on GB300 (E. Latkin, "Twofold fast summation", 2013).

The twofold sum of x (or dot of x and y) is a pair (value, error): value is
the floating-point sum in the kernels' order and error collects the rounding
errors of its additions (and, for dots, of the products), so that
value + error approximates the exact result (Overview; Example 1).

``twofold`` is the thin binding over the C-ABI library ``libtwofold.so``
(built from ``csrc/``); importing this package does not load it, so that
``inputs`` (seeded synthetic data) is usable without a GPU.  The first call
into ``twofold`` loads the library and raises if it is missing.
"""
__all__ = ["twofold", "inputs"]
