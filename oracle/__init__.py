"""FP64 CPU oracle of the explicit diffuse-interface step (test
infrastructure only: tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs).  The product path never imports it."""
from .oracle import OracleGrid, build, load, material_struct  # noqa: F401
