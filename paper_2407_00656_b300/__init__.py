"""HGKS hot path for one B300: Python binding over the libhgks C ABI.

Importing the package loads nothing; ``paper_2407_00656_b300.hgks`` loads the
shared library on first use and raises if it is missing.
"""
