"""Plain, slow FP64 CPU oracle for the thin-disk B-spline force solve (arXiv 1904.07400).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline
arm of ``bench.py`` may import anything here.  The product library never does: it shares
no code, header, table or constant generator with this package.  Every function cites the
passage of the paper it follows; where the paper is silent or ambiguous the reading taken
is stated in the function's docstring.
"""
