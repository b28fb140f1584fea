"""The oracle's thread count is a timing knob only: one thread and all of
them give bit-identical results (each output element is computed by one
loop iteration, with the same operation order)."""
import numpy as np

from oracle import oracle as O
from paper_1909_07190_gb300 import inputs as I
from paper_1909_07190_gb300 import pipelines as P


def test_one_thread_equals_all_threads():
    spec = P.harris()
    img = I.uniform_image(3, 97, 61)[0].astype(np.float64)
    n = O.num_threads()
    try:
        O.set_num_threads(1)
        assert O.num_threads() == 1
        one = O.evaluate(spec["stages"], [img], spec["outputs"])[0]
    finally:
        O.set_num_threads(n)
    assert O.num_threads() == n
    many = O.evaluate(spec["stages"], [img], spec["outputs"])[0]
    assert np.array_equal(one, many)
