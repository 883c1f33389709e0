"""TEST INFRASTRUCTURE: the CPU oracle of the fractal coder (see oracle.py)."""
