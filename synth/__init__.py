"""Seeded synthetic inputs shared by the tests, the oracle checks and the bench.

This package only draws numbers.  It holds none of the sort's arithmetic (no key
transform, no comparison, no ordering): the one sort it calls, to build the
presorted distributions, is numpy's.
"""
from .gen import *  # noqa: F401,F403
