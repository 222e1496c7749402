"""tk_sketch_draw_static: the draw entry point that allocates nothing.

It serves callers that may not allocate device memory (a closed start-up
allocation phase, a framework-owned memory pool, a plugin with no allocator);
its scratch is a fixed array inside the library.  Its output must equal the
workspace-based tk_sketch_draw, on consecutive calls that reuse the same array.
This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_07329_gb300 import build
    build.build()
    from paper_2203_07329_gb300 import tikhonov
    tikhonov.lib()
    return tikhonov


def test_static_draw_matches_workspace_draw_twice(tk):
    # two calls in a row share the static scratch; the second must not see
    # anything left by the first (different seeds and sizes on purpose)
    for seed, mp, s in [(3, 1 << 18, 8192), (11, 1000, 999), (3, 1 << 18, 8192)]:
        d_ref, r_ref = tk.tk_sketch_draw(seed, mp, s)
        d_st, r_st = tk.tk_sketch_draw_static(seed, mp, s)
        assert torch.equal(d_ref, d_st)
        assert torch.equal(r_ref, r_st)
        assert r_st.numel() == s and bool((r_st[1:] > r_st[:-1]).all())


def test_static_draw_at_the_size_limit(tk):
    mp = 1 << 20
    d_ref, r_ref = tk.tk_sketch_draw(5, mp, 4096)
    d_st, r_st = tk.tk_sketch_draw_static(5, mp, 4096)
    assert torch.equal(d_ref, d_st) and torch.equal(r_ref, r_st)


def test_static_draw_rejects_oversize(tk):
    L = tk.lib()
    st = L.tk_sketch_draw_static(1, (1 << 20) + 1, 16, None, None, None)
    assert st == tk.TK_EINVAL
    assert "TK_DRAW_STATIC_MAX_MP" in tk.last_error()
