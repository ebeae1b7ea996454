"""Test helpers: build libtpt.so if needed and import the binding."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def load():
    from paper_2603_09528_gb300 import build
    build.build()
    import paper_2603_09528_gb300 as tpt
    from paper_2603_09528_gb300 import _lib
    return tpt, _lib
