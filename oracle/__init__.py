"""CPU oracle of the ADGI per-frame probe update -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product path (``paper_2301_05125_gb300``) never imports it.
"""
